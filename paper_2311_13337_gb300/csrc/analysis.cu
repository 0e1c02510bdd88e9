// Table 2 analysis metrics of the excitatory rate series (arXiv 2311.13337,
// Sec. "Analysis metrics", Table 2: mean_PLI, mean_UD_duration,
// psd_fmax_ampmax, fit_psd_slope; Sec. "Vast parameter space exploration and
// analysis" names the PLI the mean phase lag index).
//
// Input: series [P][N][T] (set-major, time fastest; the layout of
// tvbx_series_range). Each series contributes its last T' samples, T' the
// largest number <= T whose prime factors are 2, 3 and 5, so every discrete
// Fourier transform below has length T'.
//
// Sets are processed in batches of B (scratch: the analytic signals of B
// sets, B * N * T' complex floats):
//  * an_series_kernel, one CTA per (set, region): the FP64 mean of the row;
//    UP / DOWN runs against that mean (rounded to FP32); the forward DFT of
//    the mean-removed row (in place in one shared-memory buffer: the row is
//    stored digit-reversed and transformed by decimation-in-time stages of
//    radix 2, 3, 4, 5; twiddles from a host FP64 table; for even T' as a
//    complex transform of length T'/2 of the sample pairs, untangled into the
//    spectrum of the real row); the periodogram on
//    the PSD band; the analytic signal (one-sided spectrum doubled) by the
//    inverse DFT (decimation in frequency, in place, read back through the
//    digit reversal), written to scratch;
//  * an_pli_kernel, one CTA per set: time tiles of the N analytic signals in
//    shared memory; a thread owns a 4 x 4 block of region pairs and counts
//    sign(Im(z_k conj(z_j))) by comparing the two rounded products, so
//    identical signals give exactly 0;
//  * an_finalize_kernel, one CTA per set: region-mean PSD, its peak on the
//    band, the least-squares fit of log10 PSD on log10 f (FP64), the pooled
//    UP / DOWN durations.

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.h"
#include "tvbx.h"

namespace tvbx {
namespace {

constexpr int AN_MAX_T = 8192;
constexpr int AN_MAX_STAGES = 16;
constexpr int AN_THREADS = 256;
// samples per time tile of the PLI kernel: TT (64, or 32 when the tiles of
// many regions would not fit); padded row stride of a tile plane TT + 2 floats
constexpr int PLI_TT_MAX = 64;
constexpr int PLI_TT_MIN = 32;
constexpr int PLI_THREADS = 256;

struct FftPlan {
    int n;
    int n_stages;
    int radix[AN_MAX_STAGES];
    // stage s (radix[s], DIT or DIF) has L1 = radix[0] ... radix[s-1]:
    // magic[s] = ceil(2^32 / L1) (0 for L1 = 1), so idx / L1 = umulhi(idx, magic)
    uint32_t magic[AN_MAX_STAGES];
};

__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

__device__ __forceinline__ float2 twiddle(const float2* __restrict__ tw, int e, bool inv)
{
    float2 w = __ldg(tw + e);
    if (inv) w.y = -w.y;
    return w;
}

// R-point DFT v_k = sum_q w_R^{k q} u_q with w_R = exp(sg 2 pi i / R), in the
// symmetric forms (cos and sin of 2 pi / 3 and 2 pi k / 5).
template <int R>
__device__ __forceinline__ void butterfly(const float2 (&u)[R], float2 (&v)[R], float sg)
{
    if constexpr (R == 2) {
        v[0] = cadd(u[0], u[1]);
        v[1] = csub(u[0], u[1]);
    } else if constexpr (R == 4) {
        const float2 s02 = cadd(u[0], u[2]), d02 = csub(u[0], u[2]);
        const float2 s13 = cadd(u[1], u[3]), d13 = csub(u[1], u[3]);
        const float2 jd13 = make_float2(-sg * d13.y, sg * d13.x);   // (sg i) d13
        v[0] = cadd(s02, s13);
        v[1] = cadd(d02, jd13);
        v[2] = csub(s02, s13);
        v[3] = csub(d02, jd13);
    } else if constexpr (R == 3) {
        constexpr float S3 = 0.86602540378443865f;   // sin(2 pi / 3); cos(2 pi / 3) = -1/2
        const float2 t1 = cadd(u[1], u[2]), t2 = csub(u[1], u[2]);
        const float2 a0 = make_float2(fmaf(-0.5f, t1.x, u[0].x), fmaf(-0.5f, t1.y, u[0].y));
        const float bx = sg * S3 * t2.x, by = sg * S3 * t2.y;   // (sg S3) t2, times i below
        v[0] = cadd(u[0], t1);
        v[1] = make_float2(a0.x - by, a0.y + bx);
        v[2] = make_float2(a0.x + by, a0.y - bx);
    } else {
        constexpr float C1 = 0.30901699437494742f, C2 = -0.80901699437494742f;
        constexpr float S1 = 0.95105651629515357f, S2 = 0.58778525229247313f;
        const float2 t1 = cadd(u[1], u[4]), t2 = cadd(u[2], u[3]);
        const float2 t3 = csub(u[1], u[4]), t4 = csub(u[2], u[3]);
        const float2 a1 = make_float2(fmaf(C1, t1.x, fmaf(C2, t2.x, u[0].x)), fmaf(C1, t1.y, fmaf(C2, t2.y, u[0].y)));
        const float2 a2 = make_float2(fmaf(C2, t1.x, fmaf(C1, t2.x, u[0].x)), fmaf(C2, t1.y, fmaf(C1, t2.y, u[0].y)));
        // b1 = sg (S1 t3 + S2 t4), b2 = sg (S2 t3 - S1 t4)
        const float b1x = sg * fmaf(S1, t3.x, S2 * t4.x), b1y = sg * fmaf(S1, t3.y, S2 * t4.y);
        const float b2x = sg * fmaf(S2, t3.x, -S1 * t4.x), b2y = sg * fmaf(S2, t3.y, -S1 * t4.y);
        v[0] = make_float2(u[0].x + t1.x + t2.x, u[0].y + t1.y + t2.y);
        v[1] = make_float2(a1.x - b1y, a1.y + b1x);   // a1 + i b1
        v[4] = make_float2(a1.x + b1y, a1.y - b1x);   // a1 - i b1
        v[2] = make_float2(a2.x - b2y, a2.y + b2x);   // a2 + i b2
        v[3] = make_float2(a2.x + b2y, a2.y - b2x);   // a2 - i b2
    }
}

// In-place decimation-in-time stage of radix R on a (length n, input in
// digit-reversed order): butterfly j of a block of span L = L1 R combines
// a[blk L + j + q L1], twiddled by w_L^{j q} before the R-point DFT.
template <int R>
__device__ void dit_stage(float2* a, int n, int L1, uint32_t magic, const float2* __restrict__ tw, bool inv,
                          int tws)
{
    const int L = L1 * R, nl = n / L, m = n / R;
    const float sg = inv ? 1.0f : -1.0f;
    for (int idx = threadIdx.x; idx < m; idx += blockDim.x) {
        const int blk = magic ? (int)__umulhi((uint32_t)idx, magic) : idx;   // idx / L1
        const int j = idx - blk * L1;
        float2* p = a + blk * L + j;
        float2 u[R], v[R];
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const float2 y = p[q * L1];
            u[q] = (q == 0 || j == 0) ? y : cmul(y, twiddle(tw, tws * nl * j * q, inv));
        }
        butterfly<R>(u, v, sg);
#pragma unroll
        for (int k = 0; k < R; ++k) p[k * L1] = v[k];
    }
}

// In-place decimation-in-frequency stage of radix R (natural-order input,
// span L = L1 R): the R-point DFT of a[blk L + j + q L1], each output k then
// twiddled by w_L^{j k}; after all stages the result is digit-reversed.
template <int R>
__device__ void dif_stage(float2* a, int n, int L1, uint32_t magic, const float2* __restrict__ tw, bool inv)
{
    const int L = L1 * R, nl = n / L, m = n / R;
    const float sg = inv ? 1.0f : -1.0f;
    for (int idx = threadIdx.x; idx < m; idx += blockDim.x) {
        const int blk = magic ? (int)__umulhi((uint32_t)idx, magic) : idx;   // idx / L1
        const int j = idx - blk * L1;
        float2* p = a + blk * L + j;
        float2 u[R], v[R];
#pragma unroll
        for (int q = 0; q < R; ++q) u[q] = p[q * L1];
        butterfly<R>(u, v, sg);
#pragma unroll
        for (int k = 0; k < R; ++k) p[k * L1] = (k == 0 || j == 0) ? v[k] : cmul(v[k], twiddle(tw, nl * j * k, inv));
    }
}

// Forward transform in place: a holds the input in digit-reversed order
// (a[perm[t]] = x[t]) and ends in natural order. tw holds the twiddles of a
// transform tws times longer than the plan's (every tws-th one is used).
__device__ void fft_dit(float2* a, const FftPlan& plan, const float2* __restrict__ tw, bool inv, int tws = 1)
{
    int L1 = 1;
    for (int s = 0; s < plan.n_stages; ++s) {
        const int r = plan.radix[s];
        const uint32_t mg = plan.magic[s];
        switch (r) {
        case 2: dit_stage<2>(a, plan.n, L1, mg, tw, inv, tws); break;
        case 3: dit_stage<3>(a, plan.n, L1, mg, tw, inv, tws); break;
        case 4: dit_stage<4>(a, plan.n, L1, mg, tw, inv, tws); break;
        default: dit_stage<5>(a, plan.n, L1, mg, tw, inv, tws); break;
        }
        __syncthreads();
        L1 *= r;
    }
}

// Transform in place from natural order to digit-reversed order (result t at
// a[perm[t]]): the stages in reverse radix order.
__device__ void fft_dif(float2* a, const FftPlan& plan, const float2* __restrict__ tw, bool inv)
{
    int L = plan.n;
    for (int s = plan.n_stages - 1; s >= 0; --s) {
        const int r = plan.radix[s];
        const int L1 = L / r;
        const uint32_t mg = plan.magic[s];
        switch (r) {
        case 2: dif_stage<2>(a, plan.n, L1, mg, tw, inv); break;
        case 3: dif_stage<3>(a, plan.n, L1, mg, tw, inv); break;
        case 4: dif_stage<4>(a, plan.n, L1, mg, tw, inv); break;
        default: dif_stage<5>(a, plan.n, L1, mg, tw, inv); break;
        }
        __syncthreads();
        L = L1;
    }
}

template <class T>
__device__ __forceinline__ T block_sum(T v, T* red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    T s = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    return s;
}

// One CTA per (set in batch, region). The row is held once in shared memory
// in digit-reversed order (a[perm[t]] = x_t), transformed in place forward
// (DIT, natural-order spectrum) and back (DIF, digit-reversed analytic
// signal).
//
// HALF (n even): the real row goes through a complex transform of length
// M = n / 2, z_m = x_2m + i x_2m+1 stored digit-reversed for the half plan
// (a[perm_h[m]] = z_m); with E, O the transforms of the even and odd samples,
// E_k = (Z_k + conj Z_{M-k}) / 2, O_k = -i (Z_k - conj Z_{M-k}) / 2, and
// X_k = E_k + w^k O_k, X_{M-k} = conj(E_k - w^k O_k), X_M = E_0 - O_0
// (w = exp(-2 pi i / n)); the spectrum is untangled in place, pair by pair.
template <bool HALF>
__global__ void __launch_bounds__(AN_THREADS)
an_series_kernel(const float* __restrict__ series, int N, int64_t T, FftPlan plan, FftPlan plan_h,
                 const float2* __restrict__ tw, const int* __restrict__ perm, const int* __restrict__ perm_h,
                 int band_lo, int band_n, float psd_scale, int64_t p0, float* __restrict__ psd_out,
                 int* __restrict__ ud_out, float2* __restrict__ z_out)
{
    extern __shared__ float2 an_smem[];
    __shared__ double red_d[AN_THREADS / 32];
    __shared__ int chunk_last[AN_THREADS];
    __shared__ int warp_last[AN_THREADS / 32];
    __shared__ int red_i[4][AN_THREADS / 32];
    const int n = plan.n, M = n / 2;
    float2* a = an_smem;
    const int b = blockIdx.x / N, k = blockIdx.x - b * N;
    const float* row = series + ((p0 + b) * (int64_t)N + k) * T + (T - n);
    double s = 0.0;
    if constexpr (HALF) {
        for (int m = threadIdx.x; m < M; m += blockDim.x) {
            const float x0 = row[2 * m], x1 = row[2 * m + 1];
            a[__ldg(perm_h + m)] = make_float2(x0, x1);
            s += (double)x0 + (double)x1;
        }
    } else {
        for (int t = threadIdx.x; t < n; t += blockDim.x) {
            const float x = row[t];
            a[__ldg(perm + t)] = make_float2(x, 0.0f);
            s += (double)x;
        }
    }
    const float theta = (float)(block_sum(s, red_d) / (double)n);
    // sample t of the raw row
    auto raw = [&](int t) -> float {
        if constexpr (HALF) {
            const float2 v = a[__ldg(perm_h + (t >> 1))];
            return (t & 1) ? v.y : v.x;
        } else {
            return a[__ldg(perm + t)].x;
        }
    };

    // UP / DOWN: runs between consecutive transitions (a transition at t >= 1
    // where the state differs from t - 1); thread c scans [c0, c1)
    const int per = (n + blockDim.x - 1) / blockDim.x;
    const int c0 = threadIdx.x * per, c1 = min(n, c0 + per);
    int first = -1, last = -1, nu = 0, su = 0, nd = 0, sd = 0;
    const int tb = max(c0, 1);
    bool was = tb < c1 ? raw(tb - 1) > theta : false;   // the state at tb - 1
    for (int t = tb; t < c1; ++t) {
        const bool up = raw(t) > theta;
        if (up != was) {
            if (last >= 0) {   // complete run [last, t) in state `was`
                if (was) { ++nu; su += t - last; } else { ++nd; sd += t - last; }
            }
            if (first < 0) first = t;
            last = t;
        }
        was = up;
    }
    // the run that ends at this chunk's first transition starts at the last
    // transition of the nearest preceding chunk that has one: an exclusive
    // max-scan over the chunks finds it
    chunk_last[threadIdx.x] = last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int pv = first >= 0 ? (int)threadIdx.x : -1;
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, pv, o);
        if (lane >= o) pv = max(pv, v);
    }
    if (lane == 31) warp_last[warp] = pv;
    __syncthreads();
    int prev_chunk = __shfl_up_sync(0xffffffffu, pv, 1);
    if (lane == 0) prev_chunk = -1;
    for (int w = 0; w < warp; ++w) prev_chunk = max(prev_chunk, warp_last[w]);
    if (first >= 0 && prev_chunk >= 0) {
        const int prev = chunk_last[prev_chunk];
        if (raw(prev) > theta) { ++nu; su += first - prev; } else { ++nd; sd += first - prev; }
    }
    // the four counts summed over the CTA in one pass (thread 0 writes them)
    for (int o = 16; o > 0; o >>= 1) {
        nu += __shfl_xor_sync(0xffffffffu, nu, o);
        su += __shfl_xor_sync(0xffffffffu, su, o);
        nd += __shfl_xor_sync(0xffffffffu, nd, o);
        sd += __shfl_xor_sync(0xffffffffu, sd, o);
    }
    if (lane == 0) { red_i[0][warp] = nu; red_i[1][warp] = su; red_i[2][warp] = nd; red_i[3][warp] = sd; }
    __syncthreads();   // also: the raw row was read above
    if (threadIdx.x == 0) {
        int tot[4] = {0, 0, 0, 0};
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
            for (int c = 0; c < 4; ++c) tot[c] += red_i[c][w];
        int* u = ud_out + ((int64_t)b * N + k) * 4;
        u[0] = tot[0]; u[1] = tot[1]; u[2] = tot[2]; u[3] = tot[3];
    }
    float* pr = psd_out + ((int64_t)b * N + k) * band_n;
    if constexpr (HALF) {
        for (int i = threadIdx.x; i < M; i += blockDim.x) a[i] = make_float2(a[i].x - theta, a[i].y - theta);
        __syncthreads();
        fft_dit(a, plan_h, tw, false, 2);
        // untangle pairs (i, M - i); periodogram of the band bins; analytic
        // weights h_0 = h_M = 1, h_i = 2 for 0 < i < M, 0 above M
        for (int i = threadIdx.x; i <= M / 2; i += blockDim.x) {
            if (i == 0) {
                const float2 z0 = a[0];
                a[0] = make_float2(z0.x + z0.y, 0.0f);
                a[M] = make_float2(z0.x - z0.y, 0.0f);
                continue;
            }
            const float2 zk = a[i], zm = a[M - i];
            const float2 e = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));   // (Z_i + conj Z_{M-i}) / 2
            const float2 o = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));  // -i (Z_i - conj Z_{M-i}) / 2
            const float2 t = cmul(__ldg(tw + i), o);
            const float2 xk = cadd(e, t);
            const float2 xm = make_float2(e.x - t.x, t.y - e.y);                         // conj(e - t)
            if (i >= band_lo && i < band_lo + band_n) pr[i - band_lo] = psd_scale * fmaf(xk.x, xk.x, xk.y * xk.y);
            if (M - i != i && M - i >= band_lo && M - i < band_lo + band_n)
                pr[M - i - band_lo] = psd_scale * fmaf(xm.x, xm.x, xm.y * xm.y);
            a[i] = make_float2(2.0f * xk.x, 2.0f * xk.y);
            a[M - i] = make_float2(2.0f * xm.x, 2.0f * xm.y);
        }
        for (int i = M + 1 + threadIdx.x; i < n; i += blockDim.x) a[i] = make_float2(0.0f, 0.0f);
        __syncthreads();
    } else {
        // mean-removed row
        for (int t = threadIdx.x; t < n; t += blockDim.x) a[t].x -= theta;
        __syncthreads();
        fft_dit(a, plan, tw, false);
        for (int i = threadIdx.x; i < band_n; i += blockDim.x) {
            const float2 v = a[band_lo + i];
            pr[i] = psd_scale * fmaf(v.x, v.x, v.y * v.y);
        }
        __syncthreads();   // the band is read before the spectrum is overwritten
        // analytic signal: spectrum times h (h_0 = 1, h_i = 2 below n/2, h_{n/2} = 1, 0 above)
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            float h = 0.0f;
            if (i == 0 || 2 * i == n) h = 1.0f;
            else if (2 * i < n) h = 2.0f;
            const float2 v = a[i];
            a[i] = make_float2(h * v.x, h * v.y);
        }
        __syncthreads();
    }
    fft_dif(a, plan, tw, true);
    const float inv_n = 1.0f / (float)n;
    float2* zr = z_out + ((int64_t)b * N + k) * n;
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        const float2 v = a[__ldg(perm + t)];
        zr[t] = make_float2(v.x * inv_n, v.y * inv_n);
    }
}

__device__ __forceinline__ uint64_t mul_f32x2(uint64_t a, uint64_t b)
{
    uint64_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
// sign(p - q) summed over both lanes, by comparison: the packed products are
// not subtracted, because a packed subtraction of two packed products may be
// contracted into a fused multiply-add (observed), which leaves the rounding
// error of one product instead of an exact 0 for identical signals. For
// distinct finite p and q, p - q is never 0, so the comparison is sign(p - q).
__device__ __forceinline__ int sign_diff2(uint64_t p, uint64_t q)
{
    const float p0 = __uint_as_float((uint32_t)p), p1 = __uint_as_float((uint32_t)(p >> 32));
    const float q0 = __uint_as_float((uint32_t)q), q1 = __uint_as_float((uint32_t)(q >> 32));
    return (p0 > q0) - (p0 < q0) + (p1 > q1) - (p1 < q1);
}

// One CTA per set: mean over k < j of |mean_t sign(Im(z_k conj(z_j)))|.
// The tile holds the real and imaginary parts in separate planes, time
// fastest, so one 8-byte load gives two consecutive samples and the packed
// two-lane FP32 products handle two samples of a pair per instruction (each
// lane rounds like the scalar product).
template <int PLI_TT>
__global__ void __launch_bounds__(PLI_THREADS)
an_pli_kernel(const float2* __restrict__ z_all, int N, int n, float* __restrict__ pli_out)
{
    constexpr int PLI_TS = PLI_TT + 2;
    // planes [2][(r mod 4) * NB + r / 4][PLI_TS]: the rows a half-warp reads
    // together (4 apart in r) are adjacent, and the stride (2 mod 32 words)
    // puts their 8-byte pieces in distinct banks
    extern __shared__ float tile[];
    __shared__ float red[PLI_THREADS / 32];
    const int b = blockIdx.x;
    const float2* z = z_all + (int64_t)b * N * n;
    const int NB = (N + 3) / 4, NR = NB * 4;
    float* TX = tile;
    float* TY = tile + NR * PLI_TS;
    const int nbp = NB * (NB + 1) / 2;
    float acc = 0.0f;
    for (int base = 0; base < nbp; base += blockDim.x) {
        const int bp = base + threadIdx.x;
        int bk = 0, bj = 0;
        if (bp < nbp) {   // block pair (bk <= bj), row by row
            int rem = bp;
            while (rem >= NB - bk) { rem -= NB - bk; ++bk; }
            bj = bk + rem;
        }
        int cnt[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) cnt[u][v] = 0;
        for (int t0 = 0; t0 < n; t0 += PLI_TT) {
            const int tl = min(PLI_TT, n - t0);
            __syncthreads();
            for (int i = threadIdx.x; i < NR * PLI_TT; i += blockDim.x) {
                const int r = i / PLI_TT, t = i - r * PLI_TT;
                const float2 v = (r < N && t < tl) ? z[(int64_t)r * n + t0 + t] : make_float2(0.0f, 0.0f);
                const int o = ((r & 3) * NB + (r >> 2)) * PLI_TS + t;
                TX[o] = v.x;
                TY[o] = v.y;
            }
            __syncthreads();
            if (bp < nbp) {
                // padded samples are 0 and add sign(0) = 0
                for (int t = 0; t < PLI_TT; t += 2) {
                    uint64_t xk[4], yk[4], xj[4], yj[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        xk[u] = *reinterpret_cast<const uint64_t*>(TX + (u * NB + bk) * PLI_TS + t);
                        yk[u] = *reinterpret_cast<const uint64_t*>(TY + (u * NB + bk) * PLI_TS + t);
                        xj[u] = *reinterpret_cast<const uint64_t*>(TX + (u * NB + bj) * PLI_TS + t);
                        yj[u] = *reinterpret_cast<const uint64_t*>(TY + (u * NB + bj) * PLI_TS + t);
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u)
#pragma unroll
                        for (int v = 0; v < 4; ++v) {
                            // Im(z_k conj(z_j)) = y_k x_j - x_k y_j, each product rounded
                            cnt[u][v] += sign_diff2(mul_f32x2(yk[u], xj[v]), mul_f32x2(xk[u], yj[v]));
                        }
                }
            }
        }
        if (bp < nbp) {
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    const int kk = bk * 4 + u, jj = bj * 4 + v;
                    if (kk < jj && jj < N) acc += (float)abs(cnt[u][v]) / (float)n;
                }
        }
    }
    const float tot = block_sum(acc, red);
    if (threadIdx.x == 0) pli_out[b] = N > 1 ? tot / (float)(N * (N - 1) / 2) : __int_as_float(0x7fc00000);
}

// One CTA per set: PSD mean over regions, peak, fit; UP / DOWN means.
__global__ void __launch_bounds__(AN_THREADS)
an_finalize_kernel(const float* __restrict__ psd, const int* __restrict__ ud, const float* __restrict__ pli, int N,
                   int band_lo, int band_n, double df, double dt_ms, int64_t p0, float* __restrict__ out)
{
    extern __shared__ float an_psd[];   // [band_n]
    __shared__ double red_d[4][AN_THREADS / 32];
    __shared__ float s_best[AN_THREADS];
    __shared__ int s_besti[AN_THREADS];
    __shared__ int s_pos;
    const int b = blockIdx.x;
    const float* pb = psd + (int64_t)b * N * band_n;
    for (int i = threadIdx.x; i < band_n; i += blockDim.x) {
        float s = 0.0f;
        for (int k = 0; k < N; ++k) s += pb[(int64_t)k * band_n + i];
        an_psd[i] = s / (float)N;
    }
    if (threadIdx.x == 0) s_pos = 1;
    __syncthreads();
    // peak: largest value, ties to the lower frequency
    float best = -INFINITY;
    int bi = -1;
    for (int i = threadIdx.x; i < band_n; i += blockDim.x)
        if (an_psd[i] > best) { best = an_psd[i]; bi = i; }
    s_best[threadIdx.x] = best;
    s_besti[threadIdx.x] = bi;
    // least squares of log10 PSD on log10 f (FP64)
    double su = 0.0, sv = 0.0, suu = 0.0, suv = 0.0;
    for (int i = threadIdx.x; i < band_n; i += blockDim.x) {
        const float pv = an_psd[i];
        if (!(pv > 0.0f)) { s_pos = 0; continue; }
        const double u = log10((double)(band_lo + i) * df), v = log10((double)pv);
        su += u; sv += v; suu += u * u; suv += u * v;
    }
    su = block_sum(su, red_d[0]);
    sv = block_sum(sv, red_d[1]);
    suu = block_sum(suu, red_d[2]);
    suv = block_sum(suv, red_d[3]);
    if (threadIdx.x == 0) {
        float bv = -INFINITY;
        int bix = -1;
        for (int t = 0; t < (int)blockDim.x; ++t)
            if (s_besti[t] >= 0 && (s_best[t] > bv || (s_best[t] == bv && s_besti[t] < bix))) {
                bv = s_best[t];
                bix = s_besti[t];
            }
        int64_t nu = 0, suL = 0, nd = 0, sdL = 0;
        for (int k = 0; k < N; ++k) {
            const int* u = ud + ((int64_t)b * N + k) * 4;
            nu += u[0]; suL += u[1]; nd += u[2]; sdL += u[3];
        }
        const float nan = __int_as_float(0x7fc00000);
        float* o = out + (p0 + b) * (int64_t)TVBX_AN_COUNT;
        o[TVBX_AN_MEAN_PLI] = pli[b];
        o[TVBX_AN_PSD_FMAX] = bix >= 0 ? (float)((double)(band_lo + bix) * df) : nan;
        o[TVBX_AN_PSD_AMPMAX] = bix >= 0 ? bv : nan;
        const double nb = (double)band_n;
        const double den = nb * suu - su * su;
        if (band_n >= 2 && s_pos && den != 0.0) {
            const double slope = (nb * suv - su * sv) / den;
            o[TVBX_AN_PSD_A] = (float)(-slope);
            o[TVBX_AN_PSD_B] = (float)pow(10.0, (sv - slope * su) / nb);
        } else {
            o[TVBX_AN_PSD_A] = nan;
            o[TVBX_AN_PSD_B] = nan;
        }
        o[TVBX_AN_UP_MS] = nu ? (float)((double)suL * dt_ms / (double)nu) : nan;
        o[TVBX_AN_DOWN_MS] = nd ? (float)((double)sdL * dt_ms / (double)nd) : nan;
        o[TVBX_AN_N_UP] = (float)nu;
        o[TVBX_AN_UP_SAMPLES] = (float)suL;
        o[TVBX_AN_N_DOWN] = (float)nd;
        o[TVBX_AN_DOWN_SAMPLES] = (float)sdL;
    }
}

// ---------------------------------------------------------------------------
// phFCD (Sec. "Output": the phase functional connectivity dynamics of the
// BOLD series; Deco et al. 2017): phases of the band-limited analytic
// signals, phase-coherence matrices dFC_kj(t) = cos(theta_k - theta_j), and
// the cosine similarity of their upper triangles for every t1 < t2. With unit
// phasors u_k(t), the dot product of two triangles is
//   ((|sum_k u_k(t1) u_k(t2)|^2 - N) + (|sum_k u_k(t1) conj u_k(t2)|^2 - N)) / 4,
// so a pair of times costs two complex sums over the regions.
// ---------------------------------------------------------------------------
constexpr int PF_TILE = 64;
constexpr int PF_THREADS = 256;

// One CTA per (set in batch, region): unit phasors of the band-limited
// analytic signal of the region's BOLD series, U[b][t][k] for the T' kept
// samples.
__global__ void __launch_bounds__(AN_THREADS)
an_phase_kernel(const float* __restrict__ bold, int N, int64_t P, int64_t Tb, FftPlan plan,
                const float2* __restrict__ tw, const int* __restrict__ perm, int band_lo, int band_hi, int discard,
                int64_t p0, float2* __restrict__ U)
{
    extern __shared__ float2 an_smem[];
    __shared__ double red_d[AN_THREADS / 32];
    const int n = plan.n, Tp = n - 2 * discard;
    float2* a = an_smem;   // the series in digit-reversed order, transformed in place
    const int b = blockIdx.x / N, k = blockIdx.x - b * N;
    const int64_t NP = (int64_t)N * P;
    const float* col = bold + (Tb - n) * NP + (int64_t)k * P + p0 + b;
    double s = 0.0;
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        const float x = col[(int64_t)t * NP];
        a[__ldg(perm + t)] = make_float2(x, 0.0f);
        s += (double)x;
    }
    const float mean = (float)(block_sum(s, red_d) / (double)n);
    for (int t = threadIdx.x; t < n; t += blockDim.x) a[t].x -= mean;
    __syncthreads();
    fft_dit(a, plan, tw, false);
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const float h = (i >= band_lo && i <= band_hi) ? 2.0f : 0.0f;
        a[i] = make_float2(h * a[i].x, h * a[i].y);
    }
    __syncthreads();
    fft_dif(a, plan, tw, true);
    float2* Ub = U + (int64_t)b * Tp * N;
    for (int t = threadIdx.x; t < Tp; t += blockDim.x) {
        const float2 v = a[__ldg(perm + t + discard)];
        const float r = hypotf(v.x, v.y);
        Ub[(int64_t)t * N + k] = r > 0.0f ? make_float2(v.x / r, v.y / r) : make_float2(1.0f, 0.0f);
    }
}

// One CTA per (tile pair ta <= tc of 64 x 64 times, set in batch). Tiles are
// stored region-major in shared memory; thread (m, q) owns times
// ta*64 + q + 16 i and tc*64 + m + 16 j (i, j < 4), so a half-warp reads 16
// consecutive 8-byte phasors.
__global__ void __launch_bounds__(PF_THREADS)
an_phfcd_kernel(const float2* __restrict__ U, int N, int Tp, int64_t p0, int64_t M2, float* __restrict__ out)
{
    extern __shared__ float2 pf_smem[];
    float2* Ua = pf_smem;                       // [N][64]
    float2* Uc = pf_smem + (size_t)N * PF_TILE;  // [N][64]
    __shared__ float nrm_a[PF_TILE], nrm_c[PF_TILE];
    const int nt = (Tp + PF_TILE - 1) / PF_TILE;
    int ta = 0, rem = blockIdx.x;
    while (rem >= nt - ta) { rem -= nt - ta; ++ta; }
    const int tc = ta + rem;
    const int b = blockIdx.y;
    const float2* Ub = U + (int64_t)b * Tp * N;
    for (int i = threadIdx.x; i < PF_TILE * N; i += blockDim.x) {
        const int r = i / N, k = i - r * N;
        const int t1 = ta * PF_TILE + r, t2 = tc * PF_TILE + r;
        Ua[k * PF_TILE + r] = t1 < Tp ? Ub[(int64_t)t1 * N + k] : make_float2(0.0f, 0.0f);
        Uc[k * PF_TILE + r] = t2 < Tp ? Ub[(int64_t)t2 * N + k] : make_float2(0.0f, 0.0f);
    }
    __syncthreads();
    // |V(t)| from S = sum_k u_k^2: |V|^2 = ((|S|^2 - N) + N^2 - N) / 4
    if (threadIdx.x < 2 * PF_TILE) {
        const int r = threadIdx.x & (PF_TILE - 1);
        const float2* T = threadIdx.x < PF_TILE ? Ua : Uc;
        float sx = 0.0f, sy = 0.0f;
        for (int k = 0; k < N; ++k) {
            const float2 u = T[k * PF_TILE + r];
            sx += u.x * u.x - u.y * u.y;
            sy += 2.0f * u.x * u.y;
        }
        const float fN = (float)N;
        const float v2 = 0.25f * (fmaf(sx, sx, sy * sy) - fN + fN * fN - fN);
        (threadIdx.x < PF_TILE ? nrm_a : nrm_c)[r] = sqrtf(fmaxf(v2, 0.0f));
    }
    __syncthreads();
    const int q = threadIdx.x >> 4, m = threadIdx.x & 15;
    float ax[4][4], ay[4][4], bx[4][4], by[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) ax[i][j] = ay[i][j] = bx[i][j] = by[i][j] = 0.0f;
    for (int k = 0; k < N; ++k) {
        float2 ua[4], uc[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            ua[i] = Ua[k * PF_TILE + q + 16 * i];
            uc[i] = Uc[k * PF_TILE + m + 16 * i];
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                // A += ua uc, B += ua conj(uc)
                ax[i][j] = fmaf(ua[i].x, uc[j].x, fmaf(-ua[i].y, uc[j].y, ax[i][j]));
                ay[i][j] = fmaf(ua[i].x, uc[j].y, fmaf(ua[i].y, uc[j].x, ay[i][j]));
                bx[i][j] = fmaf(ua[i].x, uc[j].x, fmaf(ua[i].y, uc[j].y, bx[i][j]));
                by[i][j] = fmaf(ua[i].y, uc[j].x, fmaf(-ua[i].x, uc[j].y, by[i][j]));
            }
    }
    const float fN = (float)N;
    float* o = out + (p0 + b) * M2;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int ra = q + 16 * i, rc = m + 16 * j;
            const int t1 = ta * PF_TILE + ra, t2 = tc * PF_TILE + rc;
            if (t1 < t2 && t2 < Tp) {
                const float dot = 0.25f * ((fmaf(ax[i][j], ax[i][j], ay[i][j] * ay[i][j]) - fN) +
                                           (fmaf(bx[i][j], bx[i][j], by[i][j] * by[i][j]) - fN));
                const int64_t e = (int64_t)t1 * Tp - (int64_t)t1 * (t1 + 1) / 2 + (t2 - t1 - 1);
                o[e] = dot / (nrm_a[ra] * nrm_c[rc]);
            }
        }
}

int smooth_length(int64_t n)
{
    for (int64_t m = std::min<int64_t>(n, AN_MAX_T); m > 0; --m) {
        int64_t r = m;
        for (int f : {2, 3, 5})
            while (r % f == 0) r /= f;
        if (r == 1) return (int)m;
    }
    return 0;
}

bool make_plan(int n, FftPlan& p)
{
    p.n = n;
    p.n_stages = 0;
    int r = n;
    // radix 5s, then 3s, then 4s, then a final 2
    for (int f : {5, 3, 4, 2}) {
        while (r % f == 0) {
            if (p.n_stages == AN_MAX_STAGES) return false;
            p.radix[p.n_stages++] = f;
            r /= f;
        }
    }
    if (r != 1) return false;
    uint64_t L1 = 1;
    for (int s = 0; s < p.n_stages; ++s) {
        // idx < 2^13 and L1 < 2^13: floor(idx * ceil(2^32 / L1) / 2^32) = floor(idx / L1)
        p.magic[s] = L1 == 1 ? 0u : (uint32_t)((((uint64_t)1 << 32) + L1 - 1) / L1);
        L1 *= (uint64_t)p.radix[s];
    }
    return true;
}

// Digit reversal of the plan: the decimation-in-time stages (radix[0] first)
// take x_t at position perm[t], and the decimation-in-frequency stages leave
// output t at perm[t]. With t = sum_k d_k W_k in the number system whose
// least significant digit has radix radix[m-1] (W_0 = 1, W_{k+1} = W_k
// radix[m-1-k]), perm[t] = sum_k d_{m-1-k} V_k with V_0 = 1,
// V_{k+1} = V_k radix[k].
std::vector<int> digit_reversal(const FftPlan& p)
{
    const int m = p.n_stages;
    std::vector<int> perm(p.n);
    for (int t = 0; t < p.n; ++t) {
        int d[AN_MAX_STAGES];
        int rem = t;
        for (int k = 0; k < m; ++k) {
            const int r = p.radix[m - 1 - k];
            d[k] = rem % r;
            rem /= r;
        }
        int v = 0, w = 1;
        for (int k = 0; k < m; ++k) {
            v += d[m - 1 - k] * w;
            w *= p.radix[k];
        }
        perm[t] = v;
    }
    return perm;
}

#define ACK(call, what)                                                                              \
    do {                                                                                             \
        cudaError_t e_ = (call);                                                                     \
        if (e_ == cudaErrorMemoryAllocation) return report_error(TVBX_E_OOM, "%s: out of memory", what); \
        if (e_ != cudaSuccess) return report_error(TVBX_E_CUDA, "%s: %s", what, cudaGetErrorString(e_)); \
    } while (0)

struct AnScratch {
    std::vector<void*> ptrs;
    cudaStream_t s;
    explicit AnScratch(cudaStream_t st) : s(st) {}
    template <class T> cudaError_t get(T** p, size_t n)
    {
        void* q = nullptr;
        cudaError_t e = cudaMallocAsync(&q, sizeof(T) * (n ? n : 1), s);
        if (e == cudaSuccess) {
            ptrs.push_back(q);
            *p = static_cast<T*>(q);
        }
        return e;
    }
    ~AnScratch()
    {
        for (void* q : ptrs) cudaFreeAsync(q, s);
    }
};

// Copy stream and events of a host-input analysis (released when the call
// returns; work still queued completes first). Before the release, the
// compute stream s waits for everything queued on the copy stream, so the
// staging buffers, freed on s afterwards, outlive every copy into them even
// when the call returns early on an error.
struct HostPipe {
    cudaStream_t s = nullptr;
    cudaStream_t cs = nullptr;
    cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};   // start, ready[2], free[2]
    ~HostPipe()
    {
        if (cs) {
            cudaEvent_t done = nullptr;
            if (cudaEventCreateWithFlags(&done, cudaEventDisableTiming) == cudaSuccess) {
                if (cudaEventRecord(done, cs) == cudaSuccess) cudaStreamWaitEvent(s, done, 0);
                cudaEventDestroy(done);
            } else {
                cudaStreamSynchronize(cs);
            }
        }
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
        if (cs) cudaStreamDestroy(cs);
    }
};

// Whether p is ordinary host memory (pageable or pinned) rather than memory
// a kernel can read.
bool is_host_pointer(const void* p)
{
    cudaPointerAttributes pa;
    if (cudaPointerGetAttributes(&pa, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return true;
    }
    return pa.type == cudaMemoryTypeHost || pa.type == cudaMemoryTypeUnregistered;
}

}  // namespace
}  // namespace tvbx

using namespace tvbx;

extern "C" tvbx_status tvbx_series_analysis(const float* series, int32_t n_regions, int64_t n_sets, int64_t n_samples,
                                            double dt_ms, float* out, int32_t* n_used, void* cuda_stream)
{
    const int N = n_regions;
    const int64_t P = n_sets, T = n_samples;
    if (!series || !out) return report_error(TVBX_E_INVALID_ARG, "NULL series or out");
    if (N < 1 || N > 752 || P < 1 || T < 2)
        return report_error(TVBX_E_INVALID_ARG, "need 1 <= n_regions <= 752, n_sets >= 1, n_samples >= 2");
    if (!(dt_ms > 0.0) || !std::isfinite(dt_ms)) return report_error(TVBX_E_INVALID_ARG, "dt_ms must be > 0");
    const int n = smooth_length(T);
    FftPlan plan;
    if (n < 2 || !make_plan(n, plan)) return report_error(TVBX_E_INVALID_ARG, "no transform length for %lld samples", (long long)T);
    // PSD band [1, 100] Hz: bins 1 <= i < n/2 with f_i = i / (n dt) in the band
    const double dt_s = dt_ms * 1e-3;
    int band_lo = -1, band_hi = -1;
    for (int i = 1; 2 * i < n; ++i) {
        const double f = (double)i / ((double)n * dt_s);
        if (f >= 1.0 && f <= 100.0) {
            if (band_lo < 0) band_lo = i;
            band_hi = i;
        }
    }
    const int band_n = band_lo < 0 ? 0 : band_hi - band_lo + 1;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    // batch of sets: analytic signals of B sets in at most ~2 GiB, B a whole
    // number of waves of the phase-lag kernel (one CTA per set) when the
    // budget allows, so no SM runs more of its CTAs than another
    const int64_t per_set = (int64_t)N * n * 8;
    int64_t B = std::max<int64_t>(1, std::min<int64_t>(P, ((int64_t)1 << 31) / std::max<int64_t>(per_set, 1)));
    const size_t pli_row = sizeof(float) * 2 * (size_t)((N + 3) / 4 * 4);
    const bool wide_tiles = pli_row * (PLI_TT_MAX + 2) <= 64 * 1024;
    const size_t smem_pli = pli_row * (size_t)((wide_tiles ? PLI_TT_MAX : PLI_TT_MIN) + 2);
    if (smem_pli > 200 * 1024) return report_error(TVBX_E_INVALID_ARG, "too many regions for the PLI tile");
    auto pli_kernel = wide_tiles ? an_pli_kernel<PLI_TT_MAX> : an_pli_kernel<PLI_TT_MIN>;
    ACK(cudaFuncSetAttribute(pli_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_pli),
        "analysis shared memory");
    {
        int dev = 0, sms = 0, per_sm = 0;
        ACK(cudaGetDevice(&dev), "device");
        ACK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "device");
        ACK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pli_kernel, PLI_THREADS, smem_pli),
            "occupancy");
        const int64_t wave = (int64_t)sms * std::max(per_sm, 1);
        if (B < P && B >= wave) B = B / wave * wave;
    }
    std::vector<float2> htw(n);
    for (int e = 0; e < n; ++e) {
        const double ang = -2.0 * 3.14159265358979323846 * (double)e / (double)n;
        htw[e] = make_float2((float)std::cos(ang), (float)std::sin(ang));
    }
    AnScratch scr(s);
    float2 *tw, *z;
    float *psd, *pli;
    int* ud;
    ACK(scr.get(&tw, n), "analysis twiddles");
    int* perm;
    ACK(scr.get(&perm, n), "analysis digit reversal");
    const std::vector<int> hperm = digit_reversal(plan);
    ACK(cudaMemcpyAsync(perm, hperm.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s), "analysis digit reversal");
    // even lengths: the forward transform as a complex one of half the length
    FftPlan plan_h = plan;
    const bool half = n % 2 == 0 && n >= 4 && make_plan(n / 2, plan_h);
    int* perm_h = perm;
    if (half) {
        ACK(scr.get(&perm_h, n / 2), "analysis digit reversal");
        const std::vector<int> hperm_h = digit_reversal(plan_h);
        ACK(cudaMemcpyAsync(perm_h, hperm_h.data(), sizeof(int) * (n / 2), cudaMemcpyHostToDevice, s),
            "analysis digit reversal");
    }
    ACK(scr.get(&z, (size_t)B * N * n), "analysis signals");
    ACK(scr.get(&psd, (size_t)B * N * std::max(band_n, 1)), "analysis PSD");
    ACK(scr.get(&pli, (size_t)B), "analysis PLI");
    ACK(scr.get(&ud, (size_t)B * N * 4), "analysis UP/DOWN");
    ACK(cudaMemcpyAsync(tw, htw.data(), sizeof(float2) * n, cudaMemcpyHostToDevice, s), "analysis twiddles");
    const size_t smem_series = sizeof(float2) * (size_t)n;
    auto series_kernel = half ? an_series_kernel<true> : an_series_kernel<false>;
    ACK(cudaFuncSetAttribute(series_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_series),
        "analysis shared memory");
    const size_t smem_fin = sizeof(float) * (size_t)std::max(band_n, 1);
    ACK(cudaFuncSetAttribute(an_finalize_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_fin),
        "analysis shared memory");
    const float psd_scale = (float)(2.0 * dt_s / (double)n * 1e6);   // kHz^2 -> Hz^2, one-sided
    const double df = 1.0 / ((double)n * dt_s);
    // host input: batch b + 1 is copied on a second stream into one of two
    // staging buffers while batch b is analysed on s
    const bool host_in = is_host_pointer(series);
    HostPipe hp;
    hp.s = s;
    float* stage[2] = {nullptr, nullptr};
    if (host_in) {
        ACK(scr.get(&stage[0], (size_t)B * N * T), "analysis staging");
        ACK(scr.get(&stage[1], (size_t)B * N * T), "analysis staging");
        ACK(cudaStreamCreateWithFlags(&hp.cs, cudaStreamNonBlocking), "analysis copy stream");
        for (cudaEvent_t& e : hp.ev) ACK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "analysis events");
        ACK(cudaEventRecord(hp.ev[0], s), "analysis events");   // the staging buffers exist
        ACK(cudaStreamWaitEvent(hp.cs, hp.ev[0], 0), "analysis events");
    }
    int64_t batch = 0;
    for (int64_t p0 = 0; p0 < P; p0 += B, ++batch) {
        const int64_t nb = std::min<int64_t>(B, P - p0);
        const float* in = series;
        int64_t in_p0 = p0;
        const int slot = (int)(batch & 1);
        if (host_in) {
            if (batch >= 2) ACK(cudaStreamWaitEvent(hp.cs, hp.ev[3 + slot], 0), "analysis events");
            ACK(cudaMemcpyAsync(stage[slot], series + p0 * N * T, sizeof(float) * (size_t)(nb * N * T),
                                cudaMemcpyHostToDevice, hp.cs),
                "analysis series upload");
            ACK(cudaEventRecord(hp.ev[1 + slot], hp.cs), "analysis events");
            ACK(cudaStreamWaitEvent(s, hp.ev[1 + slot], 0), "analysis events");
            in = stage[slot];
            in_p0 = 0;
        }
        note_launch(3);
        series_kernel<<<(unsigned)(nb * N), AN_THREADS, smem_series, s>>>(in, N, T, plan, plan_h, tw, perm, perm_h,
                                                                        band_lo, band_n, psd_scale, in_p0, psd,
                                                                        ud, z);
        ACK(cudaGetLastError(), "analysis series");
        if (host_in) ACK(cudaEventRecord(hp.ev[3 + slot], s), "analysis events");   // the slot was read
        pli_kernel<<<(unsigned)nb, PLI_THREADS, smem_pli, s>>>(z, N, n, pli);
        ACK(cudaGetLastError(), "analysis PLI");
        an_finalize_kernel<<<(unsigned)nb, AN_THREADS, smem_fin, s>>>(psd, ud, pli, N, band_lo, band_n, df, dt_ms,
                                                                       p0, out);
        ACK(cudaGetLastError(), "analysis finalize");
    }
    if (n_used) *n_used = n;
    return TVBX_OK;
}

extern "C" tvbx_status tvbx_phfcd(const float* bold, int32_t n_regions, int64_t n_sets, int64_t n_tr, double tr_s,
                                  double f_lo_hz, double f_hi_hz, int32_t discard, float* out, int32_t* n_used,
                                  void* cuda_stream)
{
    const int N = n_regions;
    const int64_t P = n_sets;
    if (!bold || !out) return report_error(TVBX_E_INVALID_ARG, "NULL bold or out");
    if (N < 2 || N > 200 || P < 1 || n_tr < 2 || discard < 0)
        return report_error(TVBX_E_INVALID_ARG, "need 2 <= n_regions <= 200, n_sets >= 1, n_tr >= 2, discard >= 0");
    if (!(tr_s > 0.0) || !std::isfinite(tr_s) || !(f_lo_hz <= f_hi_hz))
        return report_error(TVBX_E_INVALID_ARG, "need tr_s > 0 and f_lo_hz <= f_hi_hz");
    const int n = smooth_length(n_tr);
    FftPlan plan;
    if (n < 2 || !make_plan(n, plan)) return report_error(TVBX_E_INVALID_ARG, "no transform length for %lld samples", (long long)n_tr);
    const int Tp = n - 2 * discard;
    if (Tp < 2) return report_error(TVBX_E_INVALID_ARG, "fewer than 2 samples left after discarding %d at each end", discard);
    int band_lo = n, band_hi = -1;   // empty unless a bin 0 < i < n/2 has its frequency in the band
    for (int i = 1; 2 * i < n; ++i) {
        const double f = (double)i / ((double)n * tr_s);
        if (f >= f_lo_hz && f <= f_hi_hz) {
            band_lo = std::min(band_lo, i);
            band_hi = std::max(band_hi, i);
        }
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int64_t per_set = (int64_t)Tp * N * 8;
    const int64_t B = std::max<int64_t>(1, std::min<int64_t>(P, ((int64_t)1 << 30) / std::max<int64_t>(per_set, 1)));
    std::vector<float2> htw(n);
    for (int e = 0; e < n; ++e) {
        const double ang = -2.0 * 3.14159265358979323846 * (double)e / (double)n;
        htw[e] = make_float2((float)std::cos(ang), (float)std::sin(ang));
    }
    AnScratch scr(s);
    float2 *tw, *U;
    ACK(scr.get(&tw, n), "phFCD twiddles");
    int* perm;
    ACK(scr.get(&perm, n), "phFCD digit reversal");
    const std::vector<int> hperm = digit_reversal(plan);
    ACK(cudaMemcpyAsync(perm, hperm.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s), "phFCD digit reversal");
    ACK(scr.get(&U, (size_t)B * Tp * N), "phFCD phasors");
    ACK(cudaMemcpyAsync(tw, htw.data(), sizeof(float2) * n, cudaMemcpyHostToDevice, s), "phFCD twiddles");
    const size_t smem_phase = sizeof(float2) * (size_t)n;
    ACK(cudaFuncSetAttribute(an_phase_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_phase),
        "phFCD shared memory");
    const size_t smem_pf = sizeof(float2) * 2 * (size_t)N * PF_TILE;
    if (smem_pf > 200 * 1024) return report_error(TVBX_E_INVALID_ARG, "too many regions for the phFCD tiles");
    ACK(cudaFuncSetAttribute(an_phfcd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_pf),
        "phFCD shared memory");
    const int nt = (Tp + PF_TILE - 1) / PF_TILE;
    const int64_t M2 = (int64_t)Tp * (Tp - 1) / 2;
    for (int64_t p0 = 0; p0 < P; p0 += B) {
        const int64_t nb = std::min<int64_t>(B, P - p0);
        note_launch(2);
        an_phase_kernel<<<(unsigned)(nb * N), AN_THREADS, smem_phase, s>>>(bold, N, P, n_tr, plan, tw, perm, band_lo,
                                                                          band_hi, discard, p0, U);
        ACK(cudaGetLastError(), "phFCD phases");
        an_phfcd_kernel<<<dim3((unsigned)(nt * (nt + 1) / 2), (unsigned)nb), PF_THREADS, smem_pf, s>>>(U, N, Tp, p0,
                                                                                                       M2, out);
        ACK(cudaGetLastError(), "phFCD");
    }
    if (n_used) *n_used = Tp;
    return TVBX_OK;
}

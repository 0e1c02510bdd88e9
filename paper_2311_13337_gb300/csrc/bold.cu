// Balloon-Windkessel BOLD signal of the simulated excitatory rates
// (arXiv 2311.13337, Sec. "Output": a Balloon-Windkessel kernel, Stephan et
// al. 2007, turns the simulated activity into BOLD series for comparison with
// fMRI).
//
// Model (Friston et al. 2000; Stephan et al. 2007), drive z = E rate in kHz,
// time in seconds:
//   ds/dt = z - kappa s - gamma (f - 1),  df/dt = s,
//   tau dv/dt = f - v^(1/alpha),
//   tau dq/dt = f E(f) / E0 - v^(1/alpha) q / v,  E(f) = 1 - (1 - E0)^(1/f),
//   y = V0 (k1 (1 - q) + k2 (1 - q/v) + k3 (1 - v)).
// One thread per (region, set) integrates forward Euler with the step of the
// rate samples. The state is kept as deviations from rest (f - 1, v - 1,
// q - 1) and the powers are written as functions of those deviations
// (series for small arguments, log1p / expm1 beyond), so FP32 resolves the
// small excursions a drive of a few Hz causes (about 1e-3 of the resting
// values) instead of rounding them against 1, and a zero drive keeps the
// resting state exactly.
//
// Layouts: series [T][N][P] (consecutive threads read consecutive sets), BOLD
// [T / decim][N][P], state [4][N][P] = s, f - 1, v - 1, q - 1.

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <cmath>

#include "internal.h"
#include "tvbx.h"

namespace tvbx {
namespace {

struct BoldDev {
    float kappa, gamma, inv_tau, inv_alpha, r_E0, lnE, V0, k1, k2, k3, dt;   // r_E0 = (1 - E0) / E0
    float ca[8];   // binomial coefficients C(1/alpha, k), k = 1 .. 8
    float v_series;   // |v - 1| up to which the binomial series is used (0: never)
};

// (1 + v)^a - 1 for |v| <= v_series: the binomial series sum_k C(a, k) v^k to
// degree 8 (Horner); v_series is chosen on the host so that the rest of the
// series stays below 1e-8 of the first term (exact for integer a <= 8).
// Beyond it, expm1(a log1p(v)).
static __device__ __forceinline__ float pow1p_m1(float v, const BoldDev& c)
{
    if (fabsf(v) <= c.v_series) {
        float h = c.ca[7];
#pragma unroll
        for (int k = 6; k >= 0; --k) h = fmaf(h, v, c.ca[k]);
        return h * v;
    }
    return expm1f(log1pf(v) * c.inv_alpha);
}

// e^x - 1 for |x| <= 1/4 by its Taylor series to degree 8 (the rest is below
// 4.4e-11 of the first term: about x^8 / 9!), else expm1f
static __device__ __forceinline__ float expm1_small(float x)
{
    if (fabsf(x) <= 0.25f) {
        float h = 1.0f / 40320.0f;                 // 1/8!
        h = fmaf(h, x, 1.0f / 5040.0f);            // 1/7!
        h = fmaf(h, x, 1.0f / 720.0f);             // 1/6!
        h = fmaf(h, x, 1.0f / 120.0f);             // 1/5!
        h = fmaf(h, x, 1.0f / 24.0f);              // 1/4!
        h = fmaf(h, x, 1.0f / 6.0f);               // 1/3!
        h = fmaf(h, x, 0.5f);                      // 1/2!
        h = fmaf(h, x, 1.0f);
        return h * x;
    }
    return expm1f(x);
}

// 1 / x by the SM's approximate reciprocal (about 1 ulp; x is the blood
// volume 1 + (v - 1), near 1, so no denormals arise)
static __device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__global__ void bold_kernel(const float* __restrict__ series, int64_t NP, int64_t T, int decim, BoldDev c,
                            float* __restrict__ state, int reset, float* __restrict__ out)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= NP) return;
    float s = 0.0f, ft = 0.0f, vt = 0.0f, qt = 0.0f;
    if (state && !reset) {
        s = state[i];
        ft = state[NP + i];
        vt = state[2 * NP + i];
        qt = state[3 * NP + i];
    }
    int phase = 0;
    int64_t o = 0;
    for (int64_t t = 0; t < T; ++t) {
        const float z = __ldg(series + t * NP + i);
        const float f = 1.0f + ft;
        const float vpa_m1 = pow1p_m1(vt, c);                                 // v^(1/alpha) - 1
        // f E(f) / E0 - 1 = ft - (1 + ft) r_E0 expm1(-ln(1 - E0) ft / f), since
        // (1 - E0)^(1/f) = (1 - E0) exp(-ln(1 - E0) ft / f): exactly 0 at rest
        // (the argument of expm1 to 2 ulp)
        const float fE_m1 = fmaf(-f * c.r_E0, expm1_small(__fdividef(-c.lnE * ft, f)), ft);
        // v^(1/alpha - 1) q - 1, with v^(1/alpha - 1) - 1 = (v^(1/alpha) - v) / v
        // = (vpa_m1 - vt) / (1 + vt) (no cancellation: vpa_m1 is about vt / alpha)
        const float vq_m1 = fmaf((vpa_m1 - vt) * rcp_approx(1.0f + vt), 1.0f + qt, qt);
        const float ds = z - c.kappa * s - c.gamma * ft;
        const float nft = fmaf(c.dt, s, ft);
        const float nvt = fmaf(c.dt * c.inv_tau, ft - vpa_m1, vt);
        const float nqt = fmaf(c.dt * c.inv_tau, fE_m1 - vq_m1, qt);
        s = fmaf(c.dt, ds, s);
        ft = nft;
        vt = nvt;
        qt = nqt;
        if (++phase == decim) {
            phase = 0;
            // 1 - q = -qt, 1 - q / v = (vt - qt) / (1 + vt), 1 - v = -vt
            out[o * NP + i] = c.V0 * (c.k3 * -vt + fmaf(c.k1, -qt, c.k2 * (vt - qt) / (1.0f + vt)));
            ++o;
        }
    }
    if (state) {
        state[i] = s;
        state[NP + i] = ft;
        state[2 * NP + i] = vt;
        state[3 * NP + i] = qt;
    }
}

// Two FP32 values in a 64-bit register pair and the packed f32x2 operations
// of sm_100-class SMs (each lane rounds like the scalar instruction).
static __device__ __forceinline__ uint64_t p2(float lo, float hi)
{
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
static __device__ __forceinline__ float2 u2(uint64_t v)
{
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
    return r;
}
static __device__ __forceinline__ uint64_t fma2(uint64_t a, uint64_t b, uint64_t c)
{
    uint64_t r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
static __device__ __forceinline__ uint64_t mul2(uint64_t a, uint64_t b)
{
    uint64_t r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
static __device__ __forceinline__ uint64_t add2(uint64_t a, uint64_t b)
{
    uint64_t r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
static __device__ __forceinline__ uint64_t sub2(uint64_t a, uint64_t b)
{
    uint64_t r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

// The same integration for two neighbouring (region, set) elements per
// thread, i and i + 1 (i even; NP even, so every sample row starts 8-byte
// aligned), in packed f32x2 arithmetic: the series of both powers run packed
// when both lanes are inside their bounds, else lane by lane; the divisions
// and the output are lane by lane.
__global__ void bold_kernel2(const float* __restrict__ series, int64_t NP, int64_t T, int decim, BoldDev c,
                             float* __restrict__ state, int reset, float* __restrict__ out)
{
    const int64_t i = 2 * (blockIdx.x * (int64_t)blockDim.x + threadIdx.x);
    if (i >= NP) return;
    float2 s0 = make_float2(0.0f, 0.0f), f0 = s0, v0 = s0, q0 = s0;
    if (state && !reset) {
        s0 = *reinterpret_cast<const float2*>(state + i);
        f0 = *reinterpret_cast<const float2*>(state + NP + i);
        v0 = *reinterpret_cast<const float2*>(state + 2 * NP + i);
        q0 = *reinterpret_cast<const float2*>(state + 3 * NP + i);
    }
    uint64_t s = p2(s0.x, s0.y), ft = p2(f0.x, f0.y), vt = p2(v0.x, v0.y), qt = p2(q0.x, q0.y);
    const uint64_t one = p2(1.0f, 1.0f), m_kappa = p2(-c.kappa, -c.kappa), m_gamma = p2(-c.gamma, -c.gamma);
    const uint64_t dt = p2(c.dt, c.dt), dtt = p2(c.dt * c.inv_tau, c.dt * c.inv_tau);
    const uint64_t m_rE0 = p2(-c.r_E0, -c.r_E0);
    uint64_t ca[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) ca[k] = p2(c.ca[k], c.ca[k]);
    int phase = 0;
    int64_t o = 0;
    for (int64_t t = 0; t < T; ++t) {
        const float2 zf = __ldg(reinterpret_cast<const float2*>(series + t * NP + i));
        const uint64_t z = p2(zf.x, zf.y);
        const uint64_t f = add2(one, ft);
        const float2 vtf = u2(vt), ftf = u2(ft), ff = u2(f);
        // v^(1/alpha) - 1
        uint64_t vpa_m1;
        if (fabsf(vtf.x) <= c.v_series && fabsf(vtf.y) <= c.v_series) {
            uint64_t h = ca[7];
#pragma unroll
            for (int k = 6; k >= 0; --k) h = fma2(h, vt, ca[k]);
            vpa_m1 = mul2(h, vt);
        } else {
            vpa_m1 = p2(pow1p_m1(vtf.x, c), pow1p_m1(vtf.y, c));
        }
        // e^x - 1 of the oxygen extraction, x = -ln(1 - E0) ft / f
        const float x0 = __fdividef(-c.lnE * ftf.x, ff.x), x1 = __fdividef(-c.lnE * ftf.y, ff.y);
        uint64_t em1;
        if (fabsf(x0) <= 0.25f && fabsf(x1) <= 0.25f) {
            const uint64_t x = p2(x0, x1);
            uint64_t h = p2(1.0f / 40320.0f, 1.0f / 40320.0f);
            h = fma2(h, x, p2(1.0f / 5040.0f, 1.0f / 5040.0f));
            h = fma2(h, x, p2(1.0f / 720.0f, 1.0f / 720.0f));
            h = fma2(h, x, p2(1.0f / 120.0f, 1.0f / 120.0f));
            h = fma2(h, x, p2(1.0f / 24.0f, 1.0f / 24.0f));
            h = fma2(h, x, p2(1.0f / 6.0f, 1.0f / 6.0f));
            h = fma2(h, x, p2(0.5f, 0.5f));
            h = fma2(h, x, one);
            em1 = mul2(h, x);
        } else {
            em1 = p2(expm1_small(x0), expm1_small(x1));
        }
        const uint64_t fE_m1 = fma2(mul2(f, m_rE0), em1, ft);
        const float2 w = u2(add2(one, vt));
        const uint64_t rv = p2(rcp_approx(w.x), rcp_approx(w.y));
        const uint64_t vq_m1 = fma2(mul2(sub2(vpa_m1, vt), rv), add2(one, qt), qt);
        const uint64_t ds = fma2(m_gamma, ft, fma2(m_kappa, s, z));
        const uint64_t nft = fma2(dt, s, ft);
        const uint64_t nvt = fma2(dtt, sub2(ft, vpa_m1), vt);
        const uint64_t nqt = fma2(dtt, sub2(fE_m1, vq_m1), qt);
        s = fma2(dt, ds, s);
        ft = nft;
        vt = nvt;
        qt = nqt;
        if (++phase == decim) {
            phase = 0;
            const float2 a = u2(vt), b = u2(qt);
            const float y0 = c.V0 * (c.k3 * -a.x + fmaf(c.k1, -b.x, c.k2 * (a.x - b.x) / (1.0f + a.x)));
            const float y1 = c.V0 * (c.k3 * -a.y + fmaf(c.k1, -b.y, c.k2 * (a.y - b.y) / (1.0f + a.y)));
            *reinterpret_cast<float2*>(out + o * NP + i) = make_float2(y0, y1);
            ++o;
        }
    }
    if (state) {
        *reinterpret_cast<float2*>(state + i) = u2(s);
        *reinterpret_cast<float2*>(state + NP + i) = u2(ft);
        *reinterpret_cast<float2*>(state + 2 * NP + i) = u2(vt);
        *reinterpret_cast<float2*>(state + 3 * NP + i) = u2(qt);
    }
}

}  // namespace
}  // namespace tvbx

using namespace tvbx;

extern "C" tvbx_status tvbx_bold_defaults(tvbx_bold_params* out)
{
    if (!out) return report_error(TVBX_E_INVALID_ARG, "NULL out");
    out->kappa = 0.65;
    out->gamma = 0.41;
    out->tau = 0.98;
    out->alpha = 0.32;
    out->E0 = 0.34;
    out->V0 = 0.02;
    out->theta0 = 40.3;
    out->r0 = 25.0;
    out->TE = 0.04;
    out->eps = 1.0;
    return TVBX_OK;
}

extern "C" tvbx_status tvbx_bold(const float* series, int32_t n_regions, int64_t n_sets, int64_t n_samples,
                                 double dt_ms, int32_t decim, const tvbx_bold_params* params, float* state,
                                 int32_t reset_state, float* bold_out, void* cuda_stream)
{
    if (!series || !bold_out) return report_error(TVBX_E_INVALID_ARG, "NULL series or bold_out");
    if (n_regions < 1 || n_sets < 1 || n_samples < 0 || decim < 1)
        return report_error(TVBX_E_INVALID_ARG, "need n_regions >= 1, n_sets >= 1, n_samples >= 0, decim >= 1");
    if (!(dt_ms > 0.0) || !std::isfinite(dt_ms)) return report_error(TVBX_E_INVALID_ARG, "dt_ms must be > 0");
    tvbx_bold_params p;
    if (params) p = *params;
    else tvbx_bold_defaults(&p);
    if (!(p.tau > 0.0) || !(p.alpha > 0.0) || !(p.E0 > 0.0 && p.E0 < 1.0))
        return report_error(TVBX_E_INVALID_ARG, "need tau > 0, alpha > 0, 0 < E0 < 1");
    BoldDev c;
    c.kappa = (float)p.kappa;
    c.gamma = (float)p.gamma;
    c.inv_tau = (float)(1.0 / p.tau);
    c.inv_alpha = (float)(1.0 / p.alpha);
    c.r_E0 = (float)((1.0 - p.E0) / p.E0);
    c.lnE = (float)std::log1p(-p.E0);
    c.V0 = (float)p.V0;
    c.k1 = (float)(4.3 * p.theta0 * p.E0 * p.TE);
    c.k2 = (float)(p.eps * p.r0 * p.E0 * p.TE);
    c.k3 = (float)(1.0 - p.eps);
    c.dt = (float)(dt_ms * 1e-3);
    // binomial coefficients of (1 + v)^a, a = 1 / alpha, and the largest
    // |v| (a power of 2 from 1/4 down) at which the series beyond degree 8
    // stays below 1e-8 of its first term a |v|
    {
        const double a = 1.0 / p.alpha;
        double C[41];
        C[0] = 1.0;
        for (int k = 1; k <= 40; ++k) C[k] = C[k - 1] * (a - (k - 1)) / k;
        for (int k = 0; k < 8; ++k) c.ca[k] = (float)C[k + 1];
        c.v_series = 0.0f;
        for (double vm = 0.25; vm >= 1.0 / 1024.0; vm *= 0.5) {
            double tail = 0.0, pw = std::pow(vm, 9);
            for (int k = 9; k <= 40; ++k, pw *= vm) tail += std::fabs(C[k]) * pw;
            if (tail <= 1e-8 * std::fabs(a) * vm) {
                c.v_series = (float)vm;
                break;
            }
        }
    }
    const int64_t NP = (int64_t)n_regions * n_sets;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    note_launch();
    // two elements per thread when every row of series, BOLD and state starts
    // 8-byte aligned (NP even, 8-byte aligned buffers), else one
    const bool pair = NP % 2 == 0 && (uintptr_t)series % 8 == 0 && (uintptr_t)bold_out % 8 == 0 &&
                      (!state || (uintptr_t)state % 8 == 0);
    if (pair)
        bold_kernel2<<<(unsigned)((NP / 2 + 255) / 256), 256, 0, s>>>(series, NP, n_samples, decim, c, state,
                                                                      reset_state, bold_out);
    else
        bold_kernel<<<(unsigned)((NP + 255) / 256), 256, 0, s>>>(series, NP, n_samples, decim, c, state, reset_state,
                                                                bold_out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return report_error(TVBX_E_CUDA, "BOLD: %s", cudaGetErrorString(e));
    return TVBX_OK;
}

// Device-side model of the tvbx engine (arXiv 2311.13337): Philox noise, the
// transfer function with its first and second derivatives, and the Euler
// update of one (set, region) pair. Included by every simulation kernel.
//
//   Eq. 1  T dnu_mu/dt = (F_mu - nu_mu) + 1/2 sum c_{lambda eta} d2F_mu/dnu_lambda dnu_eta
//   Eq. 2  T dc_{lambda eta}/dt = delta F_lambda (1/T - F_eta)/N_lambda
//          + (F_lambda - nu_lambda)(F_eta - nu_eta)
//          + sum_mu (dF_lambda/dnu_mu c_{eta mu} + dF_eta/dnu_mu c_{lambda mu}) - 2 c_{lambda eta}
//   Eq. 3  dW/dt = -W/tau_w + b nu_e + a (mu_V - E_L)/tau_w
//   Eq. 5  F_mu(nu_e + g sum_j u_kj nu_e,j(t - tau_kj) + wNoise OU + cF_mu,e,
//               nu_i + cF_mu,i, W_mu)
// with the Zerlaut 2018 template for F and the Table 1 threshold polynomial.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace tvbx {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of the 4-word
// S-box with multipliers 0xD2511F53 / 0xCD9E8D57 and key increments
// 0x9E3779B9 / 0xBB67AE85 between rounds.
// ---------------------------------------------------------------------------
static __device__ __forceinline__ uint4 philox4x32_10(uint4 x, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        const uint32_t hi_a = __umulhi(0xD2511F53u, x.x), lo_a = 0xD2511F53u * x.x;
        const uint32_t hi_b = __umulhi(0xCD9E8D57u, x.z), lo_b = 0xCD9E8D57u * x.z;
        x = make_uint4(hi_b ^ x.y ^ k0, lo_b, hi_a ^ x.w ^ k1, lo_a);
    }
    return x;
}

// Standard normal for counter (step, region, set or 0, 0): Box-Muller on the
// first two words, u1 = (x0 + 1) 2^-32 in (0, 1], u2 = x1 2^-32.
static __device__ __forceinline__ float std_normal(uint64_t seed, uint32_t n, uint32_t k, uint32_t p)
{
    const uint4 x = philox4x32_10(make_uint4(n, k, p, 0u), (uint32_t)seed, (uint32_t)(seed >> 32));
    const float two_m32 = 2.3283064365386963e-10f;
    const float u1 = fmaf((float)x.x, two_m32, two_m32);
    const float u2 = (float)x.y * two_m32;
    return sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2);
}

// ---------------------------------------------------------------------------
// Second-order jets in the synaptic event rates (a, b) = (f_e, f_i).
// ---------------------------------------------------------------------------
struct J {
    float v, a, b, aa, ab, bb;
};

static __device__ __forceinline__ J jadd(const J& x, const J& y)
{
    return J{x.v + y.v, x.a + y.a, x.b + y.b, x.aa + y.aa, x.ab + y.ab, x.bb + y.bb};
}
static __device__ __forceinline__ J jaffine(const J& x, float s, float c)
{
    return J{fmaf(s, x.v, c), s * x.a, s * x.b, s * x.aa, s * x.ab, s * x.bb};
}
// c0 + c1 x + c2 y + c3 z for jets x, y, z
static __device__ __forceinline__ J jlin3(float c0, float c1, const J& x, float c2, const J& y, float c3,
                                   const J& z)
{
    J r;
    r.v = fmaf(c1, x.v, fmaf(c2, y.v, fmaf(c3, z.v, c0)));
    r.a = fmaf(c1, x.a, fmaf(c2, y.a, c3 * z.a));
    r.b = fmaf(c1, x.b, fmaf(c2, y.b, c3 * z.b));
    r.aa = fmaf(c1, x.aa, fmaf(c2, y.aa, c3 * z.aa));
    r.ab = fmaf(c1, x.ab, fmaf(c2, y.ab, c3 * z.ab));
    r.bb = fmaf(c1, x.bb, fmaf(c2, y.bb, c3 * z.bb));
    return r;
}
static __device__ __forceinline__ J jmul(const J& x, const J& y)
{
    J r;
    r.v = x.v * y.v;
    r.a = fmaf(x.a, y.v, x.v * y.a);
    r.b = fmaf(x.b, y.v, x.v * y.b);
    r.aa = fmaf(x.aa, y.v, fmaf(2.0f * x.a, y.a, x.v * y.aa));
    r.ab = fmaf(x.ab, y.v, fmaf(x.a, y.b, fmaf(x.b, y.a, x.v * y.ab)));
    r.bb = fmaf(x.bb, y.v, fmaf(2.0f * x.b, y.b, x.v * y.bb));
    return r;
}
// f(x) from f, f', f'' at x.v
static __device__ __forceinline__ J jchain(const J& x, float f0, float f1, float f2)
{
    J r;
    r.v = f0;
    r.a = f1 * x.a;
    r.b = f1 * x.b;
    r.aa = fmaf(f2 * x.a, x.a, f1 * x.aa);
    r.ab = fmaf(f2 * x.a, x.b, f1 * x.ab);
    r.bb = fmaf(f2 * x.b, x.b, f1 * x.bb);
    return r;
}
// Hardware approximations (PTX rcp/sqrt/ex2 .approx, flush-to-zero): at most
// a few ulp, far below the tolerances of the method.
static __device__ __forceinline__ float fast_rcp(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
static __device__ __forceinline__ float fast_rsqrt(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
static __device__ __forceinline__ float fast_exp(float x)   // e^x = 2^(x log2 e)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x * 1.44269504088896341f));
    return y;
}

// erfc(x) and 2/sqrt(pi) exp(-x^2). For x >= 0, erfc(x) = exp(-x^2) erfcx(x)
// with erfcx(x) ~= t sum c_i t^i, t = 1/(1 + x/2): a least-squares fit of the
// scaled complementary error function in t (fit_erfc.py; relative error
// 1.4e-8 in FP64, 3e-7 in float32). For x < 0, erfc(x) = 2 - erfc(-x).
static __device__ __forceinline__ void erfc_gauss(float x, float& erfc_x, float& gauss)
{
    const float ax = fabsf(x);
    const float e = fast_exp(-x * x);
    const float t = fast_rcp(fmaf(0.5f, ax, 1.0f));
    float r = 4.289677442e-02f;
    r = fmaf(r, t, -2.332135664e-01f);
    r = fmaf(r, t, +4.903904936e-01f);
    r = fmaf(r, t, -4.509691237e-01f);
    r = fmaf(r, t, +1.292146894e-01f);
    r = fmaf(r, t, -5.783515171e-02f);
    r = fmaf(r, t, +9.306424758e-02f);
    r = fmaf(r, t, +1.753847072e-01f);
    r = fmaf(r, t, +2.468781125e-01f);
    r = fmaf(r, t, +2.820940294e-01f);
    r = fmaf(r, t, +2.820947918e-01f);
    const float ec = e * (r * t);
    erfc_x = x < 0.0f ? 2.0f - ec : ec;
    gauss = 1.12837916709551257f * e;
}

static __device__ __forceinline__ J jrcp(const J& x)
{
    const float q = fast_rcp(x.v);
    const float q2 = q * q;
    return jchain(x, q, -q2, 2.0f * q2 * q);
}

// Transfer function of one population (Eq. 5, Zerlaut 2018 template, Table 1
// polynomial P) at synaptic event rates fe = K_e nu_e + floor and
// fi = K_i nu_i + floor (kHz), leak reversal E_L (mV) and adaptation W (pA).
// Returns F (kHz) with its derivatives in (fe, fi); muV receives mu_V (mV).
static __device__ __forceinline__ J transfer(const DevModel& m, const float* __restrict__ P, float E_L,
                                             float W, float fe, float fi, float& muV_out)
{
    const float qe = m.qe, qi = m.qi;
    // mean conductance and membrane potential: mu_G = g_L + qe fe + qi fi,
    // mu_V = (qe E_e fe + qi E_i fi + g_L E_L - W) / mu_G
    const float muG = fmaf(qe, fe, fmaf(qi, fi, m.g_L));
    const float r = fast_rcp(muG);
    const float r2 = r * r;
    const float num = fmaf(qe * m.E_e, fe, fmaf(qi * m.E_i, fi, fmaf(m.g_L, E_L, -W)));
    const float muV = num * r;
    muV_out = muV;
    // u = d mu_V / d fe = U_e tau_e and w = d mu_V / d fi = U_i tau_i, with
    // their closed-form derivatives (mu_V is a ratio of affine functions)
    const float u = qe * (m.E_e - muV) * r;
    const float w = qi * (m.E_i - muV) * r;
    const float s = fmaf(qe, w, qi * u);
    const J jmuV{muV, u, w, -2.0f * qe * u * r, -s * r, -2.0f * qi * w * r};
    const float cu = 2.0f * qe * r2 * fmaf(2.0f * qi, u, qe * w);
    const float cw = 2.0f * qi * r2 * fmaf(2.0f * qe, w, qi * u);
    const J ju{u, -2.0f * qe * r * u, -s * r, 6.0f * qe * qe * r2 * u, cu, cw};
    const J jw{w, -s * r, -2.0f * qi * r * w, cu, cw, 6.0f * qi * qi * r2 * w};
    // effective membrane time constant T_m = C_m / mu_G
    const float cr = m.C_m * r, cr2 = cr * r, cr3 = cr2 * r;
    const J jTm{cr, -qe * cr2, -qi * cr2, 2.0f * qe * qe * cr3, 2.0f * qe * qi * cr3, 2.0f * qi * qi * cr3};
    // shot-noise weights A_e = fe (U_e tau_e)^2, A_i = fi (U_i tau_i)^2
    const J u2 = jmul(ju, ju), w2 = jmul(jw, jw);
    const J Ae{fe * u2.v, fmaf(fe, u2.a, u2.v), fe * u2.b, fmaf(fe, u2.aa, 2.0f * u2.a),
               fmaf(fe, u2.ab, u2.b), fe * u2.bb};
    const J Ai{fi * w2.v, fi * w2.a, fmaf(fi, w2.b, w2.v), fi * w2.aa, fmaf(fi, w2.ab, w2.a),
               fmaf(fi, w2.bb, 2.0f * w2.b)};
    J De = jTm;
    De.v += m.tau_e;
    J Di = jTm;
    Di.v += m.tau_i;
    // 2 sigma_V^2 = A_e/(tau_e + T_m) + A_i/(tau_i + T_m); tau_V = (A_e + A_i) / (2 sigma_V^2)
    const J s2 = jadd(jmul(Ae, jrcp(De)), jmul(Ai, jrcp(Di)));
    // sigma_V = sqrt(s2 / 2) and 1/sigma_V from one reciprocal square root
    const float h = 0.5f * s2.v;
    const float rs = fast_rsqrt(h);
    const float rs3 = rs * rs * rs;
    const J sig = jchain(jaffine(s2, 0.5f, 0.0f), h * rs, 0.5f * rs, -0.25f * rs3);
    const J isig = jchain(jaffine(s2, 0.5f, 0.0f), rs, -0.5f * rs3, 0.75f * rs3 * rs * rs);
    const J tV = jmul(jadd(Ae, Ai), jrcp(s2));
    // normalised variables v = (V, S, Z) and the threshold polynomial in the
    // Table 1 column order (1, V, S, Z, V^2, S^2, Z^2, V S, V Z, S Z), written
    // as P0 + p.v + v^T Q v / 2 with Q = [[2P4, P7, P8], [P7, 2P5, P9], [P8, P9, 2P6]]
    const J V = jaffine(jmuV, m.inv_dmu0, -m.mu0 * m.inv_dmu0);
    const J S = jaffine(sig, m.inv_dsig0, -m.sig0 * m.inv_dsig0);
    const J Z = jaffine(tV, m.gL_over_Cm * m.inv_dtau0, -m.tau0 * m.inv_dtau0);
    const float gV = fmaf(2.0f * P[4], V.v, fmaf(P[7], S.v, fmaf(P[8], Z.v, P[1])));
    const float gS = fmaf(P[7], V.v, fmaf(2.0f * P[5], S.v, fmaf(P[9], Z.v, P[2])));
    const float gZ = fmaf(P[8], V.v, fmaf(P[9], S.v, fmaf(2.0f * P[6], Z.v, P[3])));
    const float QaV = fmaf(2.0f * P[4], V.a, fmaf(P[7], S.a, P[8] * Z.a));
    const float QaS = fmaf(P[7], V.a, fmaf(2.0f * P[5], S.a, P[9] * Z.a));
    const float QaZ = fmaf(P[8], V.a, fmaf(P[9], S.a, 2.0f * P[6] * Z.a));
    const float QbV = fmaf(2.0f * P[4], V.b, fmaf(P[7], S.b, P[8] * Z.b));
    const float QbS = fmaf(P[7], V.b, fmaf(2.0f * P[5], S.b, P[9] * Z.b));
    const float QbZ = fmaf(P[8], V.b, fmaf(P[9], S.b, 2.0f * P[6] * Z.b));
    J th;
    th.v = P[0] + fmaf(V.v, fmaf(P[4], V.v, fmaf(P[7], S.v, fmaf(P[8], Z.v, P[1]))),
                       fmaf(S.v, fmaf(P[5], S.v, fmaf(P[9], Z.v, P[2])), Z.v * fmaf(P[6], Z.v, P[3])));
    th.a = fmaf(gV, V.a, fmaf(gS, S.a, gZ * Z.a));
    th.b = fmaf(gV, V.b, fmaf(gS, S.b, gZ * Z.b));
    th.aa = fmaf(QaV, V.a, fmaf(QaS, S.a, fmaf(QaZ, Z.a, fmaf(gV, V.aa, fmaf(gS, S.aa, gZ * Z.aa)))));
    th.ab = fmaf(QaV, V.b, fmaf(QaS, S.b, fmaf(QaZ, Z.b, fmaf(gV, V.ab, fmaf(gS, S.ab, gZ * Z.ab)))));
    th.bb = fmaf(QbV, V.b, fmaf(QbS, S.b, fmaf(QbZ, Z.b, fmaf(gV, V.bb, fmaf(gS, S.bb, gZ * Z.bb)))));
    // F = erfc((V_thre - mu_V) / (sqrt(2) sigma_V)) / (2 tau_V)
    const J d{th.v - jmuV.v, th.a - jmuV.a, th.b - jmuV.b, th.aa - jmuV.aa, th.ab - jmuV.ab, th.bb - jmuV.bb};
    const J arg = jaffine(jmul(d, isig), 0.70710678118654752f, 0.0f);
    const float x = arg.v;
    float ev, g;
    erfc_gauss(x, ev, g);
    const J ec = jchain(arg, ev, -g, 2.0f * x * g);
    return jaffine(jmul(ec, jrcp(tV)), 0.5f, 0.0f);
}

// Both populations' transfer functions and their derivatives in the input
// rates (x_e, x_i) for one (set, region). out layout: [F, F_e, F_i, F_ee, F_ei, F_ii].
static __device__ __forceinline__ void transfer_x(const DevModel& m, const float* __restrict__ P, float E_L,
                                           float W, float x_e, float x_i, float out[6], float& muV)
{
    const float de = x_e > 0.0f ? m.K_e : 0.0f;
    const float di = x_i > 0.0f ? m.K_i : 0.0f;
    const float fe = fmaf(m.K_e, fmaxf(x_e, 0.0f), m.rate_floor);
    const float fi = fmaf(m.K_i, fmaxf(x_i, 0.0f), m.rate_floor);
    const J F = transfer(m, P, E_L, W, fe, fi, muV);
    out[0] = F.v;
    out[1] = de * F.a;
    out[2] = di * F.b;
    out[3] = de * de * F.aa;
    out[4] = de * di * F.ab;
    out[5] = di * di * F.bb;
}

// ---------------------------------------------------------------------------
// Contracted second-order jets for the integrator. Eq. 1 needs the Hessian of
// F only through 1/2 sum_{lambda,eta} c_{lambda eta} d2F/dnu_lambda dnu_eta,
// and Eq. 2 only its gradient, so every intermediate carries its value, its
// gradient in (fe, fi) and l = sum_ij C~_ij d_i d_j of it, with
// C~ = diag(K') C diag(K') (K' = dfe/dnu_e, dfi/dnu_i). The rules are those of
// the full jets contracted with C~: for a product l(xy) = x l(y) + y l(x)
// + 2 B(x, y), for f(x) l = f' l(x) + f'' B(x, x), with B(x, y) = grad x^T C~ grad y.
// ---------------------------------------------------------------------------
struct L4 {
    float v, a, b, l;
};
struct Cov3 {
    float aa, ab, bb;   // C~ in (fe, fi) coordinates
};

static __device__ __forceinline__ float lbil(const Cov3& c, const L4& x, const L4& y)
{
    return fmaf(x.a, fmaf(c.aa, y.a, c.ab * y.b), x.b * fmaf(c.ab, y.a, c.bb * y.b));
}
static __device__ __forceinline__ L4 ladd(const L4& x, const L4& y)
{
    return L4{x.v + y.v, x.a + y.a, x.b + y.b, x.l + y.l};
}
static __device__ __forceinline__ L4 laffine(const L4& x, float s, float c)
{
    return L4{fmaf(s, x.v, c), s * x.a, s * x.b, s * x.l};
}
static __device__ __forceinline__ L4 lmul(const Cov3& c, const L4& x, const L4& y)
{
    L4 r;
    r.v = x.v * y.v;
    r.a = fmaf(x.a, y.v, x.v * y.a);
    r.b = fmaf(x.b, y.v, x.v * y.b);
    r.l = fmaf(x.l, y.v, fmaf(x.v, y.l, 2.0f * lbil(c, x, y)));
    return r;
}
static __device__ __forceinline__ L4 lchain(const Cov3& c, const L4& x, float f0, float f1, float f2)
{
    return L4{f0, f1 * x.a, f1 * x.b, fmaf(f1, x.l, f2 * lbil(c, x, x))};
}
static __device__ __forceinline__ L4 lrcp(const Cov3& c, const L4& x)
{
    const float q = fast_rcp(x.v);
    const float q2 = q * q;
    return lchain(c, x, q, -q2, 2.0f * q2 * q);
}

// Transfer function of one population with the contracted jet (same
// template and polynomial as transfer()).
static __device__ __forceinline__ L4 transfer_lap(const DevModel& m, const float* __restrict__ P, float E_L, float W,
                                                  float fe, float fi, const Cov3& c, float& muV_out)
{
    const float qe = m.qe, qi = m.qi;
    const float muG = fmaf(qe, fe, fmaf(qi, fi, m.g_L));
    const float r = fast_rcp(muG);
    const float r2 = r * r;
    const float num = fmaf(qe * m.E_e, fe, fmaf(qi * m.E_i, fi, fmaf(m.g_L, E_L, -W)));
    const float muV = num * r;
    muV_out = muV;
    const float u = qe * (m.E_e - muV) * r;
    const float w = qi * (m.E_i - muV) * r;
    const float s = fmaf(qe, w, qi * u);
    const float cu = 2.0f * qe * r2 * fmaf(2.0f * qi, u, qe * w);
    const float cw = 2.0f * qi * r2 * fmaf(2.0f * qe, w, qi * u);
    const L4 jmuV{muV, u, w, -2.0f * r * fmaf(c.aa * qe, u, fmaf(c.ab, s, c.bb * qi * w))};
    const L4 ju{u, -2.0f * qe * r * u, -s * r, fmaf(c.aa, 6.0f * qe * qe * r2 * u, fmaf(2.0f * c.ab, cu, c.bb * cw))};
    const L4 jw{w, -s * r, -2.0f * qi * r * w, fmaf(c.aa, cu, fmaf(2.0f * c.ab, cw, c.bb * 6.0f * qi * qi * r2 * w))};
    const float cr = m.C_m * r, cr2 = cr * r, cr3 = cr2 * r;
    const L4 jTm{cr, -qe * cr2, -qi * cr2, 2.0f * cr3 * fmaf(c.aa * qe, qe, fmaf(2.0f * c.ab * qe, qi, c.bb * qi * qi))};
    const L4 u2 = lmul(c, ju, ju), w2 = lmul(c, jw, jw);
    // A_e = fe u^2 (grad fe = (1, 0)), A_i = fi w^2 (grad fi = (0, 1))
    const L4 Ae{fe * u2.v, fmaf(fe, u2.a, u2.v), fe * u2.b, fmaf(fe, u2.l, 2.0f * fmaf(c.aa, u2.a, c.ab * u2.b))};
    const L4 Ai{fi * w2.v, fi * w2.a, fmaf(fi, w2.b, w2.v), fmaf(fi, w2.l, 2.0f * fmaf(c.ab, w2.a, c.bb * w2.b))};
    L4 De = jTm;
    De.v += m.tau_e;
    L4 Di = jTm;
    Di.v += m.tau_i;
    const L4 s2 = ladd(lmul(c, Ae, lrcp(c, De)), lmul(c, Ai, lrcp(c, Di)));
    const float h = 0.5f * s2.v;
    const float rs = fast_rsqrt(h);
    const float rs3 = rs * rs * rs;
    const L4 hs = laffine(s2, 0.5f, 0.0f);
    const float bh = lbil(c, hs, hs);
    const L4 sig{h * rs, 0.5f * rs * hs.a, 0.5f * rs * hs.b, fmaf(0.5f * rs, hs.l, -0.25f * rs3 * bh)};
    const L4 isig{rs, -0.5f * rs3 * hs.a, -0.5f * rs3 * hs.b, fmaf(-0.5f * rs3, hs.l, 0.75f * rs3 * rs * rs * bh)};
    const L4 tV = lmul(c, ladd(Ae, Ai), lrcp(c, s2));
    const L4 V = laffine(jmuV, m.inv_dmu0, -m.mu0 * m.inv_dmu0);
    const L4 S = laffine(sig, m.inv_dsig0, -m.sig0 * m.inv_dsig0);
    const L4 Z = laffine(tV, m.gL_over_Cm * m.inv_dtau0, -m.tau0 * m.inv_dtau0);
    // threshold polynomial P0 + p.v + v^T Q v / 2; l = sum_ij C~_ij v_i^T Q v_j + g . l(v)
    const float gV = fmaf(2.0f * P[4], V.v, fmaf(P[7], S.v, fmaf(P[8], Z.v, P[1])));
    const float gS = fmaf(P[7], V.v, fmaf(2.0f * P[5], S.v, fmaf(P[9], Z.v, P[2])));
    const float gZ = fmaf(P[8], V.v, fmaf(P[9], S.v, fmaf(2.0f * P[6], Z.v, P[3])));
    const float QaV = fmaf(2.0f * P[4], V.a, fmaf(P[7], S.a, P[8] * Z.a));
    const float QaS = fmaf(P[7], V.a, fmaf(2.0f * P[5], S.a, P[9] * Z.a));
    const float QaZ = fmaf(P[8], V.a, fmaf(P[9], S.a, 2.0f * P[6] * Z.a));
    const float QbV = fmaf(2.0f * P[4], V.b, fmaf(P[7], S.b, P[8] * Z.b));
    const float QbS = fmaf(P[7], V.b, fmaf(2.0f * P[5], S.b, P[9] * Z.b));
    const float QbZ = fmaf(P[8], V.b, fmaf(P[9], S.b, 2.0f * P[6] * Z.b));
    const float aQa = fmaf(QaV, V.a, fmaf(QaS, S.a, QaZ * Z.a));
    const float aQb = fmaf(QbV, V.a, fmaf(QbS, S.a, QbZ * Z.a));
    const float bQb = fmaf(QbV, V.b, fmaf(QbS, S.b, QbZ * Z.b));
    L4 th;
    th.v = P[0] + fmaf(V.v, fmaf(P[4], V.v, fmaf(P[7], S.v, fmaf(P[8], Z.v, P[1]))),
                       fmaf(S.v, fmaf(P[5], S.v, fmaf(P[9], Z.v, P[2])), Z.v * fmaf(P[6], Z.v, P[3])));
    th.a = fmaf(gV, V.a, fmaf(gS, S.a, gZ * Z.a));
    th.b = fmaf(gV, V.b, fmaf(gS, S.b, gZ * Z.b));
    th.l = fmaf(c.aa, aQa, fmaf(2.0f * c.ab, aQb, fmaf(c.bb, bQb, fmaf(gV, V.l, fmaf(gS, S.l, gZ * Z.l)))));
    const L4 d{th.v - jmuV.v, th.a - jmuV.a, th.b - jmuV.b, th.l - jmuV.l};
    const L4 arg = laffine(lmul(c, d, isig), 0.70710678118654752f, 0.0f);
    const float x = arg.v;
    float ev, g;
    erfc_gauss(x, ev, g);
    const L4 ec = lchain(c, arg, ev, -g, 2.0f * x * g);
    return laffine(lmul(c, ec, lrcp(c, tV)), 0.5f, 0.0f);
}

// F, its gradient in the input rates (x_e, x_i) and sum_ij C_ij d2F/dx_i dx_j
// for the covariance C = [[Cee, Cei], [Cei, Cii]] of the pair.
static __device__ __forceinline__ void transfer_x_lap(const DevModel& m, const float* __restrict__ P, float E_L,
                                                      float W, float x_e, float x_i, float Cee, float Cei, float Cii,
                                                      float out[4], float& muV)
{
    const float de = x_e > 0.0f ? m.K_e : 0.0f;
    const float di = x_i > 0.0f ? m.K_i : 0.0f;
    const float fe = fmaf(m.K_e, fmaxf(x_e, 0.0f), m.rate_floor);
    const float fi = fmaf(m.K_i, fmaxf(x_i, 0.0f), m.rate_floor);
    const Cov3 c{de * de * Cee, de * di * Cei, di * di * Cii};
    const L4 F = transfer_lap(m, P, E_L, W, fe, fi, c, muV);
    out[0] = F.v;
    out[1] = de * F.a;
    out[2] = di * F.b;
    out[3] = F.l;
}

// Per-set parameters of the simulation kernels (11 floats, in this order).
struct SetParams {
    float g, b_e, inv_tw, ELe, ELi, a_e, wn, cFee, cFei, cFie, cFii;
};
static_assert(sizeof(SetParams) == 11 * sizeof(float), "SetParams must be 11 packed floats");

static __device__ __forceinline__ SetParams load_set_params(const float* __restrict__ prm, int64_t P, int64_t p)
{
    SetParams s;
    s.g = prm[TVBX_AXIS_G * P + p];
    s.b_e = prm[TVBX_AXIS_B_E * P + p];
    s.inv_tw = 1.0f / prm[TVBX_AXIS_TAU_W_E * P + p];
    s.ELe = prm[TVBX_AXIS_E_L_E * P + p];
    s.ELi = prm[TVBX_AXIS_E_L_I * P + p];
    s.a_e = prm[TVBX_AXIS_A_E * P + p];
    s.wn = prm[TVBX_AXIS_W_NOISE * P + p];
    s.cFee = prm[TVBX_AXIS_CF_EE * P + p];
    s.cFei = prm[TVBX_AXIS_CF_EI * P + p];
    s.cFie = prm[TVBX_AXIS_CF_IE * P + p];
    s.cFii = prm[TVBX_AXIS_CF_II * P + p];
    return s;
}

// State of one (set, region) pair.
struct PairState {
    float E, I, Cee, Cei, Cii, We, Wi;
};

// One forward-Euler step of Eq. 1-3 for one pair, from the state at step n,
// the delayed coupling sum_j u_kj E_j(n - d_kj) and the OU value at step n.
// E and I are clamped to [E_min, E_max] after the update; NaN is kept.
static __device__ __forceinline__ void euler_step(const DevModel& m, const SetParams& sp, PairState& x,
                                                  float coupling, float OU, uint32_t& flags)
{
    const float E = x.E, I = x.I, ce = x.Cee, cx = x.Cei, ci = x.Cii, We = x.We, Wi = x.Wi;
    const float exc = fmaf(sp.wn, OU, fmaf(sp.g, coupling, E));
    // F, gradient in (nu_e, nu_i), and sum c_{lambda eta} d2F/dnu_lambda dnu_eta
    float Fe[4], Fi[4], muVe, muVi;
    transfer_x_lap(m, m.P_e, sp.ELe, We, exc + sp.cFee, I + sp.cFei, ce, cx, ci, Fe, muVe);
    transfer_x_lap(m, m.P_i, sp.ELi, Wi, exc + sp.cFie, I + sp.cFii, ce, cx, ci, Fi, muVi);
    const float rT = m.inv_T;
    const float dFe = Fe[0] - E, dFi = Fi[0] - I;
    // Eq. 1
    const float dE = fmaf(0.5f, Fe[3], dFe) * rT;
    const float dI = fmaf(0.5f, Fi[3], dFi) * rT;
    // Eq. 2
    const float dCee = (Fe[0] * (rT - Fe[0]) * m.inv_Ne + dFe * dFe
                        + 2.0f * fmaf(ce, Fe[1], cx * Fe[2]) - 2.0f * ce) * rT;
    const float dCei = (dFe * dFi + fmaf(cx, Fe[1], ci * Fe[2]) + fmaf(ce, Fi[1], cx * Fi[2])
                        - 2.0f * cx) * rT;
    const float dCii = (Fi[0] * (rT - Fi[0]) * m.inv_Ni + dFi * dFi
                        + 2.0f * fmaf(cx, Fi[1], ci * Fi[2]) - 2.0f * ci) * rT;
    // Eq. 3
    const float dWe = fmaf(sp.b_e, E, (sp.a_e * (muVe - sp.ELe) - We) * sp.inv_tw);
    const float dWi = fmaf(m.b_i, I, (m.a_i * (muVi - sp.ELi) - Wi) * m.inv_tau_w_i);
    const float dt = m.dt;
    float En = fmaf(dt, dE, E), In = fmaf(dt, dI, I);
    x.Cee = fmaf(dt, dCee, ce);
    x.Cei = fmaf(dt, dCei, cx);
    x.Cii = fmaf(dt, dCii, ci);
    if (fmaxf(fabsf(x.Cee), fmaxf(fabsf(x.Cei), fabsf(x.Cii))) > m.C_div) flags |= TVBX_SET_DIVERGED;
    x.We = fmaf(dt, dWe, We);
    x.Wi = fmaf(dt, dWi, Wi);
    if (!isfinite(En) || !isfinite(In)) flags |= TVBX_SET_NONFINITE;
    if (En > m.E_max) { En = m.E_max; flags |= TVBX_SET_CLAMP_HI; }
    if (En < m.E_min) { En = m.E_min; flags |= TVBX_SET_CLAMP_LO; }
    if (In > m.E_max) { In = m.E_max; flags |= TVBX_SET_CLAMP_HI; }
    if (In < m.E_min) { In = m.E_min; flags |= TVBX_SET_CLAMP_LO; }
    x.E = En;
    x.I = In;
}

// Kahan-compensated accumulation s += v with carry c.
static __device__ __forceinline__ void kahan_add(float& s, float& c, float v)
{
    const float y = v - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}

}  // namespace tvbx

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

#include <type_traits>

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

// ---------------------------------------------------------------------------
// Lane arithmetic of the integrator. A thread integrates either one set
// (float) or two sets held in the two halves of a register pair (float2,
// FP32x2 instructions). Every operation rounds once to nearest and no product
// is ever fused into a later sum (explicit round-to-nearest operations), so a
// set's result is the same in either form and in either half of a pair.
// ---------------------------------------------------------------------------
static __device__ __forceinline__ float vfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
static __device__ __forceinline__ float vmul(float a, float b) { return __fmul_rn(a, b); }
static __device__ __forceinline__ float vadd(float a, float b) { return __fadd_rn(a, b); }
static __device__ __forceinline__ float vsub(float a, float b) { return __fsub_rn(a, b); }
// The packed forms are written in PTX (fma/mul/add/sub.rn.f32x2 on register
// pairs). The assembler fuses a packed product into a packed sum that
// consumes it even when contraction is disabled, so the integrator never
// feeds a product (vmul) into vadd or vsub: where a product meets a sum the
// code writes the fused form itself (vfma), and a product that later meets a
// sum is formed as vfma(a, b, +0), the same number as a * b except that a
// zero product is +0 (the assembler cannot turn it back into a product).
static __device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c)
{
    float2 d;
    asm("{\n\t.reg .b64 pa, pb, pc, pd;\n\t"
        "mov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\tmov.b64 pc, {%6, %7};\n\t"
        "fma.rn.f32x2 pd, pa, pb, pc;\n\tmov.b64 {%0, %1}, pd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}
static __device__ __forceinline__ float2 vmul(float2 a, float2 b)
{
    float2 d;
    asm("{\n\t.reg .b64 pa, pb, pd;\n\tmov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
        "mul.rn.f32x2 pd, pa, pb;\n\tmov.b64 {%0, %1}, pd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
static __device__ __forceinline__ float2 vadd(float2 a, float2 b)
{
    float2 d;
    asm("{\n\t.reg .b64 pa, pb, pd;\n\tmov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
        "add.rn.f32x2 pd, pa, pb;\n\tmov.b64 {%0, %1}, pd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
static __device__ __forceinline__ float2 vsub(float2 a, float2 b)
{
    float2 d;
    asm("{\n\t.reg .b64 pa, pb, pd;\n\tmov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
        "sub.rn.f32x2 pd, pa, pb;\n\tmov.b64 {%0, %1}, pd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}

template <class V> static __device__ __forceinline__ V vbc(float s);
template <> __device__ __forceinline__ float vbc<float>(float s) { return s; }
template <> __device__ __forceinline__ float2 vbc<float2>(float s) { return make_float2(s, s); }

// lane-wise maps
template <class F> static __device__ __forceinline__ float vmap(float x, F f) { return f(x); }
template <class F> static __device__ __forceinline__ float2 vmap(float2 x, F f) { return make_float2(f(x.x), f(x.y)); }
template <class F> static __device__ __forceinline__ float vmap2(float x, float y, F f) { return f(x, y); }
template <class F> static __device__ __forceinline__ float2 vmap2(float2 x, float2 y, F f)
{
    return make_float2(f(x.x, y.x), f(x.y, y.y));
}
template <class V> static __device__ __forceinline__ V vrcp(V x) { return vmap(x, [](float u) { return fast_rcp(u); }); }
template <class V> static __device__ __forceinline__ V vrsqrt(V x) { return vmap(x, [](float u) { return fast_rsqrt(u); }); }
// NaN-propagating minimum and maximum (a NaN operand gives NaN)
static __device__ __forceinline__ float fmin_nan(float a, float b)
{
    float y;
    asm("min.NaN.f32 %0, %1, %2;" : "=f"(y) : "f"(a), "f"(b));
    return y;
}
static __device__ __forceinline__ float fmax_nan(float a, float b)
{
    float y;
    asm("max.NaN.f32 %0, %1, %2;" : "=f"(y) : "f"(a), "f"(b));
    return y;
}
static __device__ __forceinline__ float lane(float x, int) { return x; }
static __device__ __forceinline__ float lane(float2 x, int i) { return i ? x.y : x.x; }
static __device__ __forceinline__ void set_lane(float& x, int, float v) { x = v; }
static __device__ __forceinline__ void set_lane(float2& x, int i, float v)
{
    if (i) x.y = v;
    else x.x = v;
}
template <class V> struct Lanes;
template <> struct Lanes<float> { static constexpr int n = 1; };
template <> struct Lanes<float2> { static constexpr int n = 2; };

// erfc(x) and 2/sqrt(pi) exp(-x^2), lane by lane in the same operations as
// erfc_gauss (the fit of the scaled complementary error function in
// t = 1/(1 + |x|/2); erfc(x) = 2 - erfc(-x) for x < 0).
template <class V>
static __device__ __forceinline__ void verfc_gauss(V x, V& erfc_x, V& gauss)
{
    const V ax = vmap(x, [](float u) { return fabsf(u); });
    const V e = vmap(vmul(vmul(x, x), vbc<V>(-1.44269504088896341f)), [](float u) {
        float y;
        asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(u));
        return y;
    });
    const V t = vrcp(vfma(vbc<V>(0.5f), ax, vbc<V>(1.0f)));
    V r = vbc<V>(4.289677442e-02f);
    r = vfma(r, t, vbc<V>(-2.332135664e-01f));
    r = vfma(r, t, vbc<V>(+4.903904936e-01f));
    r = vfma(r, t, vbc<V>(-4.509691237e-01f));
    r = vfma(r, t, vbc<V>(+1.292146894e-01f));
    r = vfma(r, t, vbc<V>(-5.783515171e-02f));
    r = vfma(r, t, vbc<V>(+9.306424758e-02f));
    r = vfma(r, t, vbc<V>(+1.753847072e-01f));
    r = vfma(r, t, vbc<V>(+2.468781125e-01f));
    r = vfma(r, t, vbc<V>(+2.820940294e-01f));
    r = vfma(r, t, vbc<V>(+2.820947918e-01f));
    const V rt = vmul(r, t);
    const V ec = vmul(e, rt);
    const V two_m = vfma(vmul(vbc<V>(-1.0f), e), rt, vbc<V>(2.0f));   // 2 - e r t, rounded once
    erfc_x = ec;
#pragma unroll
    for (int i = 0; i < Lanes<V>::n; ++i)
        if (lane(x, i) < 0.0f) set_lane(erfc_x, i, lane(two_m, i));
    gauss = vmul(vbc<V>(1.12837916709551257f), e);
}

// ---------------------------------------------------------------------------
// Contracted second-order jets of the integrator (see L4 above): value,
// gradient (a, b) in the event rates (fe, fi) and l = sum_ij C~_ij d_i d_j,
// with C~ the covariance in event-rate coordinates.
// ---------------------------------------------------------------------------
template <class V> struct CJ {
    V v, a, b, l;
};

// ---------------------------------------------------------------------------
// Reduced transfer function, for tau_e == tau_i = tau. With a_e = (E_e - mu_V)
// mu_G and a_i = (E_i - mu_V) mu_G, the Zerlaut template collapses to
//   mu_V = E_e - a_e / mu_G,  a_e = g_L (E_e - E_L) + W + q_i (E_e - E_i) f_i,
//   a_i = a_e - (E_e - E_i) mu_G,
//   sigma_V^2 = rho Q,  Q = q_e^2 f_e a_e^2 + q_i^2 f_i a_i^2,
//   rho = 1 / (2 mu_G^3 D),  D = tau mu_G + C_m,
//   tau_V = tau + C_m / mu_G,  so 1 / (2 tau_V) = phi = mu_G / (2 D),
// (q_mu = Q_mu tau), the same functions with fewer operations. rho, phi and
// tau_V depend on the inputs only through mu_G, so their jets follow from
// scalar derivatives in mu_G. The threshold polynomial is folded with the
// normalisation: (V_thre - mu_V) / sqrt(2) = c0 + c1 V + c2 S + c3 Z + c4 V^2
// + c5 S^2 + c6 Z^2 + c7 V S + c8 V Z + c9 S Z in the normalised variables
// (V, S, Z) (DevModel::cp_e, cp_i), and the erfc argument is that times
// 1/sigma_V.
// ---------------------------------------------------------------------------
// Part of the reduced transfer function that depends only on the event-rate
// pair (fe, fi) and the covariance C~, shared by the two populations when
// their inputs coincide.
template <class V> struct TFShare {
    V fe, fi;            // event rates (kHz)
    V caa, cab, cbb;     // C~
    V mu;                // mu_G
    V ga, gb, bG;        // C~ grad mu_G = (ga, gb) and B(mu_G, mu_G)
    V r, r2, r3;         // powers of 1 / mu_G
    V nr;                // -1 / mu_G
    V rho, rho1, rhol;   // rho with d rho / d mu_G and its contraction l
    V phi, phi1, phil;   // phi = 1 / (2 tau_V) likewise
    V Zv, Zl, zr;        // Z: value, l; grad Z = zr (q_e, q_i)
    V BZZ;               // B(Z, Z)
    V SQ2;               // the part of l(Q) common to both populations
};

template <class V>
static __device__ __forceinline__ void tf_share(const DevModel& m, V fe, V fi, V caa, V cab, V cbb, TFShare<V>& s)
{
    s.fe = fe;
    s.fi = fi;
    s.caa = caa;
    s.cab = cab;
    s.cbb = cbb;
    const V mu = vfma(vbc<V>(m.qi), fi, vfma(vbc<V>(m.qe), fe, vbc<V>(m.g_L)));
    s.mu = mu;
    const V D = vfma(vbc<V>(m.tau), mu, vbc<V>(m.C_m));
    const V q = vrcp(vmul(mu, D));           // 1 / (mu_G D), one reciprocal for both
    const V r = vmul(D, q), rD = vmul(mu, q);
    s.ga = vfma(caa, vbc<V>(m.qe), vmul(cab, vbc<V>(m.qi)));
    s.gb = vfma(cab, vbc<V>(m.qe), vmul(cbb, vbc<V>(m.qi)));
    s.bG = vfma(vbc<V>(m.qe), s.ga, vmul(vbc<V>(m.qi), s.gb));
    const V r2 = vmul(r, r), r3 = vmul(r2, r);
    s.r = r;
    s.r2 = r2;
    s.r3 = r3;
    s.nr = vmul(vbc<V>(-1.0f), r);
    // rho = r^3 rD / 2; d ln rho / d mu_G = -(3 r + tau rD) = nlam;
    // rho'' = (nlam^2 + 3 r^2 + (tau rD)^2) rho
    const V hD = vmul(vbc<V>(0.5f), rD);
    const V rho = vmul(r3, hD);
    const V tDn = vmul(vbc<V>(-m.tau), rD);
    const V nlam = vfma(vbc<V>(-3.0f), r, tDn);
    s.rho = rho;
    s.rho1 = vmul(nlam, rho);
    s.rhol = vmul(vmul(vfma(nlam, nlam, vfma(tDn, tDn, vmul(vbc<V>(3.0f), r2))), rho), s.bG);
    // phi = mu_G rD / 2; phi' = C_m rD^2 / 2; phi'' = -2 tau rD phi'
    s.phi = vmul(mu, hD);
    s.phi1 = vmul(vmul(vbc<V>(m.C_m), hD), rD);
    s.phil = vmul(vmul(vmul(vbc<V>(2.0f), tDn), s.phi1), s.bG);
    // Z = z0 + z1 r: grad Z = -z1 r^2 (q_e, q_i), l(Z) = 2 z1 r^3 B(mu_G, mu_G)
    s.Zv = vfma(vbc<V>(m.z1), r, vbc<V>(m.z0));
    s.Zl = vmul(vmul(vbc<V>(m.two_z1), r3), s.bG);
    s.zr = vmul(vbc<V>(-m.z1), r2);
    s.BZZ = vmul(vmul(vbc<V>(m.z1sq), vmul(r2, r2)), s.bG);
    // 2 (caa q_i^2 b_i^2 fi + cbb q_e^2 b_e^2 fe)
    s.SQ2 = vfma(vmul(caa, fi), vbc<V>(m.sq_i), vmul(vmul(cbb, fe), vbc<V>(m.sq_e)));
}

// One population (POP 0 = e, 1 = i): F with its gradient in (fe, fi) and
// l(F); muV receives mu_V. alpha = g_L (E_e - E_L) + W.
// Coefficient k of population POP's folded polynomial, read as a member (a
// kernel-parameter constant, not a load through a pointer).
template <int POP> static __device__ __forceinline__ float cpoly(const DevModel& m, int k);
template <> __device__ __forceinline__ float cpoly<0>(const DevModel& m, int k) { return m.cp_e[k]; }
template <> __device__ __forceinline__ float cpoly<1>(const DevModel& m, int k) { return m.cp_i[k]; }

template <int POP, class V>
static __device__ __forceinline__ CJ<V> tf_pop(const DevModel& m, const TFShare<V>& s, V alpha, V& muV)
{
    const V ae = vfma(vbc<V>(m.be), s.fi, alpha);
    const V ai = vfma(vbc<V>(-m.dE), s.mu, ae);
    const V aer = vmul(ae, s.r);
    muV = vfma(ae, s.nr, vbc<V>(m.E_e));   // E_e - a_e / mu_G, rounded once
    // V = (mu_V - mu0) / dmu0 = v0 - v1 a_e r
    CJ<V> Vj;
    Vj.v = vfma(vbc<V>(-m.v1), aer, vbc<V>(m.v0));
    const V r2ae = vmul(s.r2, ae);
    Vj.a = vmul(vbc<V>(m.v1qe), r2ae);
    Vj.b = vfma(vbc<V>(m.v1qi), r2ae, vmul(vbc<V>(-m.v1be), s.r));
    Vj.l = vmul(vmul(vbc<V>(-m.two_v1), s.r2), vfma(aer, s.bG, vmul(vbc<V>(-m.be), s.gb)));
    // Q = q_e^2 fe a_e^2 + q_i^2 fi a_i^2 (d a_e / d fi = b_e, d a_i / d fe = b_i)
    const V te = vmul(vbc<V>(m.ke), ae), ti = vmul(vbc<V>(m.ki), ai);
    const V fete = vmul(s.fe, te), fiti = vmul(s.fi, ti);
    CJ<V> Q;
    Q.v = vfma(fete, ae, vmul(fiti, ai));
    Q.a = vfma(te, ae, vmul(fiti, vbc<V>(m.two_bi)));
    Q.b = vfma(fete, vbc<V>(m.two_be), vmul(ti, ai));
    Q.l = vfma(vmul(vbc<V>(4.0f), s.cab), vfma(te, vbc<V>(m.be), vmul(ti, vbc<V>(m.bi))), s.SQ2);
    // sigma_V^2 = Q rho
    CJ<V> s2;
    s2.v = vmul(Q.v, s.rho);
    s2.a = vfma(Q.a, s.rho, vmul(Q.v, vmul(s.rho1, vbc<V>(m.qe))));
    s2.b = vfma(Q.b, s.rho, vmul(Q.v, vmul(s.rho1, vbc<V>(m.qi))));
    s2.l = vfma(vbc<V>(2.0f), vmul(s.rho1, vfma(Q.a, s.ga, vmul(Q.b, s.gb))),
                vfma(Q.l, s.rho, vmul(Q.v, s.rhol)));
    const V Csa = vfma(s.caa, s2.a, vmul(s.cab, s2.b));
    const V Csb = vfma(s.cab, s2.a, vmul(s.cbb, s2.b));
    const V Bs = vfma(s2.a, Csa, vmul(s2.b, Csb));
    // S = (sigma_V - sig0) / dsig0, sigma_V = s2 / sqrt(s2)
    const V rs = vrsqrt(s2.v);
    const V rs2 = vmul(rs, rs), rs3 = vmul(rs2, rs);
    const V h1 = vmul(rs, vbc<V>(m.s1h));
    CJ<V> S;
    S.v = vfma(vmul(s2.v, rs), vbc<V>(m.s1), vbc<V>(-m.s0));
    S.a = vmul(h1, s2.a);
    S.b = vmul(h1, s2.b);
    S.l = vfma(h1, s2.l, vmul(vbc<V>(-m.s1q), vmul(rs3, Bs)));
    const V BSS = vmul(vmul(h1, h1), Bs);
    // bilinear terms of the polynomial's variables
    const V CVa = vfma(s.caa, Vj.a, vmul(s.cab, Vj.b));
    const V CVb = vfma(s.cab, Vj.a, vmul(s.cbb, Vj.b));
    const V BVV = vfma(Vj.a, CVa, vmul(Vj.b, CVb));
    const V BVS = vfma(S.a, CVa, vmul(S.b, CVb));
    const V CZa = vmul(s.zr, s.ga), CZb = vmul(s.zr, s.gb);
    const V BVZ = vfma(Vj.a, CZa, vmul(Vj.b, CZb));
    const V BSZ = vfma(S.a, CZa, vmul(S.b, CZb));
    const V Za = vmul(s.zr, vbc<V>(m.qe)), Zb = vmul(s.zr, vbc<V>(m.qi));
    // d = (V_thre - mu_V) / sqrt(2) and its jet
    const V Z = s.Zv;
    const V t = vfma(vbc<V>(cpoly<POP>(m, 8)), Z, vfma(vbc<V>(cpoly<POP>(m, 7)), S.v, vfma(vbc<V>(cpoly<POP>(m, 4)), Vj.v, vbc<V>(cpoly<POP>(m, 1)))));
    const V u = vfma(vbc<V>(cpoly<POP>(m, 9)), Z, vfma(vbc<V>(cpoly<POP>(m, 5)), S.v, vbc<V>(cpoly<POP>(m, 2))));
    const V w = vfma(vbc<V>(cpoly<POP>(m, 6)), Z, vbc<V>(cpoly<POP>(m, 3)));
    CJ<V> d;
    d.v = vfma(Vj.v, t, vfma(S.v, u, vfma(Z, w, vbc<V>(cpoly<POP>(m, 0)))));
    const V gV = vfma(vbc<V>(cpoly<POP>(m, 4)), Vj.v, t);
    const V gS = vfma(vbc<V>(cpoly<POP>(m, 7)), Vj.v, vfma(vbc<V>(cpoly<POP>(m, 5)), S.v, u));
    const V gZ = vfma(vbc<V>(cpoly<POP>(m, 8)), Vj.v, vfma(vbc<V>(cpoly<POP>(m, 9)), S.v, vfma(vbc<V>(cpoly<POP>(m, 6)), Z, w)));
    d.a = vfma(gV, Vj.a, vfma(gS, S.a, vmul(gZ, Za)));
    d.b = vfma(gV, Vj.b, vfma(gS, S.b, vmul(gZ, Zb)));
    const V H = vfma(vbc<V>(cpoly<POP>(m, 4)), BVV,
                     vfma(vbc<V>(cpoly<POP>(m, 5)), BSS,
                          vfma(vbc<V>(cpoly<POP>(m, 6)), s.BZZ,
                               vfma(vbc<V>(cpoly<POP>(m, 7)), BVS, vfma(vbc<V>(cpoly<POP>(m, 8)), BVZ, vmul(vbc<V>(cpoly<POP>(m, 9)), BSZ))))));
    d.l = vfma(vbc<V>(2.0f), H, vfma(gV, Vj.l, vfma(gS, S.l, vmul(gZ, s.Zl))));
    // y = d / sigma_V, with d(1/sigma_V)/d s2 = k1 = -rs^3/2 and d2 = 3 rs^5 / 4
    const V k1 = vmul(vbc<V>(-0.5f), rs3);
    CJ<V> y;
    y.v = vmul(d.v, rs);
    const V dk = vmul(d.v, k1);
    y.a = vfma(d.a, rs, vmul(dk, s2.a));
    y.b = vfma(d.b, rs, vmul(dk, s2.b));
    const V Bds = vfma(d.a, Csa, vmul(d.b, Csb));
    const V il = vfma(k1, s2.l, vmul(vmul(vmul(vbc<V>(0.75f), rs3), rs2), Bs));
    y.l = vfma(d.l, rs, vfma(d.v, il, vmul(vmul(vbc<V>(-1.0f), rs3), Bds)));
    // erfc(y): erfc' = -g, erfc'' = 2 y g
    V ev, g;
    verfc_gauss(y.v, ev, g);
    const V ng = vmul(vbc<V>(-1.0f), g);
    const V Cya = vfma(s.caa, y.a, vmul(s.cab, y.b));
    const V Cyb = vfma(s.cab, y.a, vmul(s.cbb, y.b));
    const V Byy = vfma(y.a, Cya, vmul(y.b, Cyb));
    const V eca = vmul(ng, y.a), ecb = vmul(ng, y.b);
    const V ecl = vfma(ng, y.l, vmul(vmul(vmul(vbc<V>(2.0f), y.v), g), Byy));
    // F = erfc(y) phi
    CJ<V> F;
    F.v = vfma(ev, s.phi, vbc<V>(0.0f));   // ev phi >= 0; an fma, so no later sum absorbs it
    F.a = vfma(eca, s.phi, vmul(ev, vmul(s.phi1, vbc<V>(m.qe))));
    F.b = vfma(ecb, s.phi, vmul(ev, vmul(s.phi1, vbc<V>(m.qi))));
    F.l = vfma(vbc<V>(2.0f), vmul(s.phi1, vfma(eca, s.ga, vmul(ecb, s.gb))), vfma(ecl, s.phi, vmul(ev, s.phil)));
    return F;
}

// Input rates of one population: event rates fe = K_e max(x_e, 0) + floor,
// fi likewise, the slopes de = d fe / d x_e and di (0 where the input is
// clipped), and C~ = diag(de, di) C diag(de, di).
template <class V>
static __device__ __forceinline__ void tf_inputs(const DevModel& m, V x_e, V x_i, V ce, V cx, V ci, V& fe, V& fi,
                                                 V& de, V& di, V& caa, V& cab, V& cbb)
{
    const float Ke = m.K_e, Ki = m.K_i;
    de = vmap(x_e, [Ke](float u) { return u > 0.0f ? Ke : 0.0f; });
    di = vmap(x_i, [Ki](float u) { return u > 0.0f ? Ki : 0.0f; });
    fe = vfma(vbc<V>(Ke), vmap(x_e, [](float u) { return fmaxf(u, 0.0f); }), vbc<V>(m.rate_floor));
    fi = vfma(vbc<V>(Ki), vmap(x_i, [](float u) { return fmaxf(u, 0.0f); }), vbc<V>(m.rate_floor));
    caa = vmul(vmul(de, de), ce);
    cab = vmul(vmul(de, di), cx);
    cbb = vmul(vmul(di, di), ci);
}

// One population's transfer function as the integrator evaluates it (reduced
// form when tau_e == tau_i, else the general template): out = F, dF/dx_e,
// dF/dx_i and sum_ij C_ij d2F/dx_i dx_j; muV receives mu_V. pop: 0 = e, 1 = i.
static __device__ __forceinline__ void transfer_integrator(const DevModel& m, int pop, float E_L, float W, float x_e,
                                                           float x_i, float Cee, float Cei, float Cii, float out[4],
                                                           float& muV)
{
    if (!m.reduced) {
        transfer_x_lap(m, pop ? m.P_i : m.P_e, E_L, W, x_e, x_i, Cee, Cei, Cii, out, muV);
        return;
    }
    float fe, fi, de, di, caa, cab, cbb;
    tf_inputs(m, x_e, x_i, Cee, Cei, Cii, fe, fi, de, di, caa, cab, cbb);
    TFShare<float> sh;
    tf_share(m, fe, fi, caa, cab, cbb, sh);
    const float alpha = vadd(vfma(-m.g_L, E_L, m.gLEe), W);
    const CJ<float> F = pop ? tf_pop<1>(m, sh, alpha, muV) : tf_pop<0>(m, sh, alpha, muV);
    out[0] = F.v;
    out[1] = vmul(de, F.a);
    out[2] = vmul(di, F.b);
    out[3] = F.l;
}

// Per-set parameters of the simulation kernels (11 values, in this order).
template <class V> struct ParamsV {
    V g, b_e, inv_tw, ELe, ELi, a_e, wn, cFee, cFei, cFie, cFii;
};
using SetParams = ParamsV<float>;
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

// State of one (set, region) pair, or of two sets of one region. cWe, cWi:
// carries of the compensated Euler updates of the adaptation currents.
template <class V> struct PairV {
    V E, I, Cee, Cei, Cii, We, Wi, cWe, cWi;
};
using PairState = PairV<float>;

// Status bits (TVBX_SET_*) of each set a thread integrates, gathered over a
// chunk.
template <class V> struct Track {
    uint32_t f[Lanes<V>::n];
};
template <class V> static __device__ __forceinline__ Track<V> track_init()
{
    Track<V> t;
#pragma unroll
    for (int i = 0; i < Lanes<V>::n; ++i) t.f[i] = 0u;
    return t;
}
template <class V> static __device__ __forceinline__ uint32_t track_flags(const DevModel&, const Track<V>& t, int i)
{
    return t.f[i];
}
// Event bits of one step from the updated (unclamped) E and I and the largest
// |covariance| (NaN ignored).
static __device__ __noinline__ uint32_t step_events(const DevModel& m, float e, float i, float cm)
{
    uint32_t f = 0u;
    if (!isfinite(e) || !isfinite(i)) f |= TVBX_SET_NONFINITE;
    if (e > m.E_max || i > m.E_max) f |= TVBX_SET_CLAMP_HI;
    if (e < m.E_min || i < m.E_min) f |= TVBX_SET_CLAMP_LO;
    if (cm > m.C_div) f |= TVBX_SET_DIVERGED;
    return f;
}

// Both populations' transfer functions in the reduced form for the inputs
// (xee, xie) of the excitatory and (xei, xii) of the inhibitory population:
// F, l(F) and the gradient in the input rates (Fex = dF_e/dx_e, ...). The
// part shared by the two populations is computed once when their inputs
// coincide (the same numbers either way).
template <class V>
static __device__ __forceinline__ void pair_tf_reduced(const DevModel& m, const ParamsV<V>& sp, V We, V Wi, V ce, V cx,
                                                       V ci, V xee, V xie, V xei, V xii, CJ<V>& Fe, CJ<V>& Fi,
                                                       V& Fex, V& Fey, V& Fix, V& Fiy, V& muVe, V& muVi)
{
    V fe, fi, de, di, caa, cab, cbb;
    tf_inputs(m, xee, xie, ce, cx, ci, fe, fi, de, di, caa, cab, cbb);
    TFShare<V> sh;
    tf_share(m, fe, fi, caa, cab, cbb, sh);
    const V gLEe = vbc<V>(m.gLEe), ngL = vbc<V>(-m.g_L);
    Fe = tf_pop<0>(m, sh, vadd(vfma(ngL, sp.ELe, gLEe), We), muVe);
    const V zero = vbc<V>(0.0f);
    Fex = vfma(de, Fe.a, zero);   // products that later meet sums: see the lane arithmetic
    Fey = vfma(di, Fe.b, zero);
    // the shared part again for the inhibitory inputs (recomputed rather than
    // kept: the same numbers when the inputs coincide, and no registers held
    // across the excitatory population)
    V xei_ = xei, xii_ = xii;
#pragma unroll
    for (int i = 0; i < Lanes<V>::n; ++i) {
        float u = lane(xei_, i), w = lane(xii_, i);
        asm volatile("" : "+f"(u), "+f"(w));
        set_lane(xei_, i, u);
        set_lane(xii_, i, w);
    }
    tf_inputs(m, xei_, xii_, ce, cx, ci, fe, fi, de, di, caa, cab, cbb);
    tf_share(m, fe, fi, caa, cab, cbb, sh);
    Fi = tf_pop<1>(m, sh, vadd(vfma(ngL, sp.ELi, gLEe), Wi), muVi);
    Fix = vfma(de, Fi.a, zero);
    Fiy = vfma(di, Fi.b, zero);
}

// Both populations' transfer functions by the general template (tau_e !=
// tau_i), out of line so that its registers stay off the budget of the
// reduced form that the kernels run otherwise.
static __device__ __noinline__ void pair_tf_general(const DevModel& m, float ELe, float ELi, float We, float Wi,
                                                    float ce, float cx, float ci, float xee, float xie, float xei,
                                                    float xii, float* oe, float* oi, float& muVe, float& muVi)
{
    transfer_x_lap(m, m.P_e, ELe, We, xee, xie, ce, cx, ci, oe, muVe);
    transfer_x_lap(m, m.P_i, ELi, Wi, xei, xii, ce, cx, ci, oi, muVi);
}

// One forward-Euler step of Eq. 1-3 for one pair (or two sets of one region),
// from the state at step n, the delayed coupling sum_j u_kj E_j(n - d_kj) and
// the OU value at step n. E and I are clamped to [E_min, E_max] after the
// update (NaN kept); the events go to the tracker.
template <class V>
static __device__ __forceinline__ void pair_step(const DevModel& m, const ParamsV<V>& sp, PairV<V>& x, V coupling,
                                                 V OU, Track<V>& trk)
{
    const V E = x.E, I = x.I, ce = x.Cee, cx = x.Cei, ci = x.Cii, We = x.We, Wi = x.Wi;
    const V exc = vfma(sp.wn, OU, vfma(sp.g, coupling, E));
    const V xee = vadd(exc, sp.cFee), xie = vadd(I, sp.cFei);
    const V xei = vadd(exc, sp.cFie), xii = vadd(I, sp.cFii);
    CJ<V> Fe, Fi;
    V Fex, Fey, Fix, Fiy, muVe, muVi;
    if constexpr (std::is_same<V, float>::value) {
        if (!m.reduced) {   // general template (tau_e != tau_i)
            float oe[4], oi[4];
            pair_tf_general(m, sp.ELe, sp.ELi, We, Wi, ce, cx, ci, xee, xie, xei, xii, oe, oi, muVe, muVi);
            Fe = CJ<V>{oe[0], 0.0f, 0.0f, oe[3]};
            Fi = CJ<V>{oi[0], 0.0f, 0.0f, oi[3]};
            Fex = oe[1];
            Fey = oe[2];
            Fix = oi[1];
            Fiy = oi[2];
        } else {
            pair_tf_reduced(m, sp, We, Wi, ce, cx, ci, xee, xie, xei, xii, Fe, Fi, Fex, Fey, Fix, Fiy, muVe, muVi);
        }
    } else {
        pair_tf_reduced(m, sp, We, Wi, ce, cx, ci, xee, xie, xei, xii, Fe, Fi, Fex, Fey, Fix, Fiy, muVe, muVi);
    }
    const V one = vbc<V>(1.0f), rT = vbc<V>(m.inv_T);
    const V dFe = vsub(Fe.v, E), dFi = vsub(Fi.v, I);
    // Eq. 1
    const V dE = vmul(vfma(vbc<V>(0.5f), Fe.l, dFe), rT);
    const V dI = vmul(vfma(vbc<V>(0.5f), Fi.l, dFi), rT);
    // Eq. 2
    const V tee = vfma(cx, Fey, vmul(ce, vsub(Fex, one)));
    const V dCee = vmul(vfma(vmul(Fe.v, vsub(rT, Fe.v)), vbc<V>(m.inv_Ne), vfma(dFe, dFe, vmul(vbc<V>(2.0f), tee))), rT);
    const V dCei = vmul(vfma(dFe, dFi, vfma(ce, Fix, vfma(ci, Fey, vmul(cx, vadd(vadd(Fex, Fiy), vbc<V>(-2.0f)))))),
                        rT);
    const V tii = vfma(cx, Fix, vmul(ci, vsub(Fiy, one)));
    const V dCii = vmul(vfma(vmul(Fi.v, vsub(rT, Fi.v)), vbc<V>(m.inv_Ni), vfma(dFi, dFi, vmul(vbc<V>(2.0f), tii))), rT);
    // Eq. 3
    const V dWe = vfma(sp.b_e, E, vmul(vfma(sp.a_e, vsub(muVe, sp.ELe), vmul(vbc<V>(-1.0f), We)), sp.inv_tw));
    const V dWi = vfma(vbc<V>(m.b_i), I,
                       vmul(vfma(vbc<V>(m.a_i), vsub(muVi, sp.ELi), vmul(vbc<V>(-1.0f), Wi)), vbc<V>(m.inv_tau_w_i)));
    const V dt = vbc<V>(m.dt);
    const V En = vfma(dt, dE, E), In = vfma(dt, dI, I);
    x.Cee = vfma(dt, dCee, ce);
    x.Cei = vfma(dt, dCei, cx);
    x.Cii = vfma(dt, dCii, ci);
    // W_e, W_i relax over tau_w >> dt: a plain FP32 update stops moving once
    // dt dW falls below half an ulp of W, (tau_w / dt) 2^-24 short of the
    // equilibrium (2.5e-4 relative at 417 ms), so the increments are added
    // with a Kahan carry (the same Euler step, summed without that loss)
    const V yWe = vfma(dt, dWe, vmul(vbc<V>(-1.0f), x.cWe));
    const V tWe = vadd(We, yWe);
    x.cWe = vsub(vsub(tWe, We), yWe);
    x.We = tWe;
    const V yWi = vfma(dt, dWi, vmul(vbc<V>(-1.0f), x.cWi));
    const V tWi = vadd(Wi, yWi);
    x.cWi = vsub(vsub(tWi, Wi), yWi);
    x.Wi = tWi;
    // clamp of E and I (NaN kept); a clamp, a value that is not finite or a
    // covariance beyond C_div (all of which change or fail one of the three
    // comparisons) takes the rare path that records the event bits
    const float Emin = m.E_min, Emax = m.E_max;
#pragma unroll
    for (int i = 0; i < Lanes<V>::n; ++i) {
        const float e = lane(En, i), ii = lane(In, i);
        const float ce_ = fmin_nan(fmax_nan(e, Emin), Emax), ci_ = fmin_nan(fmax_nan(ii, Emin), Emax);
        const float cm = fmaxf(fabsf(lane(x.Cee, i)), fmaxf(fabsf(lane(x.Cei, i)), fabsf(lane(x.Cii, i))));
        set_lane(x.E, i, ce_);
        set_lane(x.I, i, ci_);
        if (!(ce_ == e && ci_ == ii && cm <= m.C_div)) trk.f[i] |= step_events(m, e, ii, cm);
    }
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

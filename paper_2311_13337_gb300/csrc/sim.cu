// Simulation kernels of the tvbx engine: Philox noise, the shared OU table,
// the transfer function with its first and second derivatives, and the
// chunked lock-step integration of all (set, region) pairs.
//
// Model (arXiv 2311.13337, Sec. "Mean Field model" and "Transfer Function"):
//   Eq. 1  T dnu_mu/dt = (F_mu - nu_mu) + 1/2 sum c_{lambda eta} d2F_mu/dnu_lambda dnu_eta
//   Eq. 2  T dc_{lambda eta}/dt = delta F_lambda (1/T - F_eta)/N_lambda
//          + (F_lambda - nu_lambda)(F_eta - nu_eta)
//          + sum_mu (dF_lambda/dnu_mu c_{eta mu} + dF_eta/dnu_mu c_{lambda mu}) - 2 c_{lambda eta}
//   Eq. 3  dW/dt = -W/tau_w + b nu_e + a (mu_V - E_L)/tau_w
//   Eq. 4  tau_OU dOU = (mu - OU) dt + sigma dW_t
//   Eq. 5  F_mu(nu_e + g sum_j u_kj nu_e,j(t - tau_kj) + wNoise OU + cF_mu,e,
//               nu_i + cF_mu,i, W_mu)
// with the Zerlaut 2018 template for F and the Table 1 threshold polynomial.
// Forward Euler (Sec. "MPI", last paragraph), temporal average of the inner
// steps (Sec. "Output").

#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace tvbx {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of the 4-word
// S-box with multipliers 0xD2511F53 / 0xCD9E8D57 and key increments
// 0x9E3779B9 / 0xBB67AE85 between rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 x, uint32_t k0, uint32_t k1)
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
__device__ __forceinline__ float std_normal(uint64_t seed, uint32_t n, uint32_t k, uint32_t p)
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

__device__ __forceinline__ J jadd(const J& x, const J& y)
{
    return J{x.v + y.v, x.a + y.a, x.b + y.b, x.aa + y.aa, x.ab + y.ab, x.bb + y.bb};
}
__device__ __forceinline__ J jaffine(const J& x, float s, float c)
{
    return J{fmaf(s, x.v, c), s * x.a, s * x.b, s * x.aa, s * x.ab, s * x.bb};
}
// c0 + c1 x + c2 y + c3 z for jets x, y, z
__device__ __forceinline__ J jlin3(float c0, float c1, const J& x, float c2, const J& y, float c3,
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
__device__ __forceinline__ J jmul(const J& x, const J& y)
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
__device__ __forceinline__ J jchain(const J& x, float f0, float f1, float f2)
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
__device__ __forceinline__ J jrcp(const J& x)
{
    const float q = __frcp_rn(x.v);
    const float q2 = q * q;
    return jchain(x, q, -q2, 2.0f * q2 * q);
}
__device__ __forceinline__ J jsqrt(const J& x)
{
    const float s = sqrtf(x.v);
    const float is = __frcp_rn(s);
    return jchain(x, s, 0.5f * is, -0.25f * is * is * is);
}

// Transfer function of one population (Eq. 5, Zerlaut 2018 template, Table 1
// polynomial P) at synaptic event rates fe = K_e nu_e + floor and
// fi = K_i nu_i + floor (kHz), leak reversal E_L (mV) and adaptation W (pA).
// Returns F (kHz) with its derivatives in (fe, fi); muV receives mu_V (mV).
__device__ __forceinline__ J transfer(const DevModel& m, const float* __restrict__ P, float E_L,
                                      float W, float fe, float fi, float& muV_out)
{
    const float qe = m.qe, qi = m.qi;
    // mean conductance and membrane potential: mu_G = g_L + qe fe + qi fi,
    // mu_V = (qe E_e fe + qi E_i fi + g_L E_L - W) / mu_G
    const float muG = fmaf(qe, fe, fmaf(qi, fi, m.g_L));
    const float r = __frcp_rn(muG);
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
    const J sig = jsqrt(jaffine(s2, 0.5f, 0.0f));
    const J tV = jmul(jadd(Ae, Ai), jrcp(s2));
    // normalised variables and the threshold polynomial (Table 1 column order:
    // 1, V, S, Z, V^2, S^2, Z^2, V S, V Z, S Z)
    const J V = jaffine(jmuV, m.inv_dmu0, -m.mu0 * m.inv_dmu0);
    const J S = jaffine(sig, m.inv_dsig0, -m.sig0 * m.inv_dsig0);
    const J Z = jaffine(tV, m.gL_over_Cm * m.inv_dtau0, -m.tau0 * m.inv_dtau0);
    const J A1 = jlin3(P[1], P[4], V, P[7], S, P[8], Z);
    const J A2 = jlin3(P[2], 0.0f, V, P[5], S, P[9], Z);
    const J A3 = jaffine(Z, P[6], P[3]);
    J th = jadd(jadd(jmul(V, A1), jmul(S, A2)), jmul(Z, A3));
    th.v += P[0];
    // F = erfc((V_thre - mu_V) / (sqrt(2) sigma_V)) / (2 tau_V)
    J d = th;
    d.v -= jmuV.v; d.a -= jmuV.a; d.b -= jmuV.b; d.aa -= jmuV.aa; d.ab -= jmuV.ab; d.bb -= jmuV.bb;
    const J arg = jaffine(jmul(d, jrcp(sig)), 0.70710678118654752f, 0.0f);
    const float x = arg.v;
    const float g = 1.12837916709551257f * expf(-x * x);  // 2/sqrt(pi) exp(-x^2)
    const J ec = jchain(arg, erfcf(x), -g, 2.0f * x * g);
    return jaffine(jmul(ec, jrcp(tV)), 0.5f, 0.0f);
}

// Both populations' transfer functions and their derivatives in the input
// rates (x_e, x_i) for one (set, region). out layout: [F, F_e, F_i, F_ee, F_ei, F_ii].
__device__ __forceinline__ void transfer_x(const DevModel& m, const float* __restrict__ P, float E_L,
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
// Initial state: E = E0, I = I0, everything else 0 (OU starts at 0).
// ---------------------------------------------------------------------------
__global__ void init_state_kernel(float* __restrict__ state, uint32_t* __restrict__ status,
                                  int64_t NP, int64_t P, float E0, float I0)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < NP * SV_COUNT;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = i / NP;
        state[i] = v == SV_E ? E0 : (v == SV_I ? I0 : 0.0f);
    }
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < P;
         p += (int64_t)gridDim.x * blockDim.x)
        status[p] = 0u;
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
template <int PB>
__global__ void __launch_bounds__(512)
sim_chunk_kernel(const __grid_constant__ SimArgs a)
{
    extern __shared__ float st[];  // [SV_COUNT][N][PB]
    const TileDev tile = a.tiles[blockIdx.x];
    const GroupDev grp = a.groups[tile.group];
    const DevModel& m = a.m;
    const int N = a.N;
    const int P = a.P;
    const int npairs = N * PB;

    for (int i = threadIdx.x; i < SV_COUNT * npairs; i += blockDim.x) {
        const int v = i / npairs, rem = i - v * npairs, k = rem / PB, q = rem - k * PB;
        st[i] = q < tile.nq ? a.state[((int64_t)v * N + k) * P + grp.p_base + tile.q0 + q] : 0.0f;
    }
    __syncthreads();

    const int q = threadIdx.x % PB;
    const int kstart = threadIdx.x / PB;
    const int kstride = blockDim.x / PB;
    const bool active = q < tile.nq;
    const int qg = tile.q0 + q;           // column in the group's ring
    const int p = grp.p_base + qg;        // internal set index

    float g = 0.f, b_e = 0.f, inv_tw = 1.f, ELe = 0.f, ELi = 0.f, a_e = 0.f, wn = 0.f;
    float cFee = 0.f, cFei = 0.f, cFie = 0.f, cFii = 0.f;
    uint32_t pn = 0u;
    if (active) {
        g = a.prm[TVBX_AXIS_G * (int64_t)P + p];
        b_e = a.prm[TVBX_AXIS_B_E * (int64_t)P + p];
        inv_tw = 1.0f / a.prm[TVBX_AXIS_TAU_W_E * (int64_t)P + p];
        ELe = a.prm[TVBX_AXIS_E_L_E * (int64_t)P + p];
        ELi = a.prm[TVBX_AXIS_E_L_I * (int64_t)P + p];
        a_e = a.prm[TVBX_AXIS_A_E * (int64_t)P + p];
        wn = a.prm[TVBX_AXIS_W_NOISE * (int64_t)P + p];
        cFee = a.prm[TVBX_AXIS_CF_EE * (int64_t)P + p];
        cFei = a.prm[TVBX_AXIS_CF_EI * (int64_t)P + p];
        cFie = a.prm[TVBX_AXIS_CF_IE * (int64_t)P + p];
        cFii = a.prm[TVBX_AXIS_CF_II * (int64_t)P + p];
        pn = (uint32_t)(a.p_offset + a.ext_index[p]);
    }
    uint32_t flags = 0u;
    const int64_t slot_stride = (int64_t)N * grp.P_g;
    const float inv_ts = 1.0f / (float)a.ts;
    const float dt = m.dt;

    for (int s = 0; s < a.n_chunk; ++s) {
        const int64_t n = a.n0 + s;
        const int slot_n = (int)(n % grp.H);
        const int slot_w = slot_n + 1 == grp.H ? 0 : slot_n + 1;
        const bool sample_now = ((n + 1) % a.ts) == 0;
        const int64_t t = (n + 1) / a.ts - 1;
        if (active) {
            for (int k = kstart; k < N; k += kstride) {
                // delayed coupling: g sum_j u_kj E_j(n - d_kj)
                float acc = 0.0f;
                const int e1 = grp.row_ptr[k + 1];
                for (int e = grp.row_ptr[k]; e < e1; ++e) {
                    const uint32_t cd = __ldg(grp.col_dly + e);
                    const int j = (int)(cd & 0xffffu);
                    int sl = slot_n - (int)(cd >> 16);
                    sl += sl < 0 ? grp.H : 0;
                    acc = fmaf(__ldg(grp.w + e), grp.ring[sl * slot_stride + (int64_t)j * grp.P_g + qg], acc);
                }
                float* sk = st + k * PB + q;
                const float E = sk[SV_E * npairs], I = sk[SV_I * npairs];
                const float ce = sk[SV_CEE * npairs], cx = sk[SV_CEI * npairs], ci = sk[SV_CII * npairs];
                const float We = sk[SV_WE * npairs], Wi = sk[SV_WI * npairs];
                float OU;
                if (a.noise_per_set) OU = sk[SV_OU * npairs];
                else OU = a.ou_table[(int64_t)s * N + k];

                const float exc = fmaf(wn, OU, fmaf(g, acc, E));
                float Fe[6], Fi[6], muVe, muVi;
                transfer_x(m, m.P_e, ELe, We, exc + cFee, I + cFei, Fe, muVe);
                transfer_x(m, m.P_i, ELi, Wi, exc + cFie, I + cFii, Fi, muVi);

                const float rT = m.inv_T;
                const float dFe = Fe[0] - E, dFi = Fi[0] - I;
                // Eq. 1
                const float dE = (dFe + 0.5f * fmaf(ce, Fe[3], fmaf(2.0f * cx, Fe[4], ci * Fe[5]))) * rT;
                const float dI = (dFi + 0.5f * fmaf(ce, Fi[3], fmaf(2.0f * cx, Fi[4], ci * Fi[5]))) * rT;
                // Eq. 2
                const float dCee = (Fe[0] * (rT - Fe[0]) * m.inv_Ne + dFe * dFe
                                    + 2.0f * fmaf(ce, Fe[1], cx * Fe[2]) - 2.0f * ce) * rT;
                const float dCei = (dFe * dFi + fmaf(cx, Fe[1], ci * Fe[2]) + fmaf(ce, Fi[1], cx * Fi[2])
                                    - 2.0f * cx) * rT;
                const float dCii = (Fi[0] * (rT - Fi[0]) * m.inv_Ni + dFi * dFi
                                    + 2.0f * fmaf(cx, Fi[1], ci * Fi[2]) - 2.0f * ci) * rT;
                // Eq. 3
                const float dWe = fmaf(b_e, E, (a_e * (muVe - ELe) - We) * inv_tw);
                const float dWi = fmaf(m.b_i, I, (m.a_i * (muVi - ELi) - Wi) * m.inv_tau_w_i);

                float En = fmaf(dt, dE, E), In = fmaf(dt, dI, I);
                sk[SV_CEE * npairs] = fmaf(dt, dCee, ce);
                sk[SV_CEI * npairs] = fmaf(dt, dCei, cx);
                sk[SV_CII * npairs] = fmaf(dt, dCii, ci);
                sk[SV_WE * npairs] = fmaf(dt, dWe, We);
                sk[SV_WI * npairs] = fmaf(dt, dWi, Wi);
                if (a.noise_per_set) {
                    const float xi = std_normal(a.seed, (uint32_t)n, (uint32_t)k, pn);
                    sk[SV_OU * npairs] = fmaf(m.ou_a, m.ou_mu - OU, fmaf(m.ou_b, xi, OU));
                }
                if (!isfinite(En) || !isfinite(In)) flags |= TVBX_SET_NONFINITE;
                if (En > m.E_max) { En = m.E_max; flags |= TVBX_SET_CLAMP_HI; }
                if (En < m.E_min) { En = m.E_min; flags |= TVBX_SET_CLAMP_LO; }
                if (In > m.E_max) { In = m.E_max; flags |= TVBX_SET_CLAMP_HI; }
                if (In < m.E_min) { In = m.E_min; flags |= TVBX_SET_CLAMP_LO; }
                sk[SV_E * npairs] = En;
                sk[SV_I * npairs] = In;
                grp.ring[slot_w * slot_stride + (int64_t)k * grp.P_g + qg] = En;

                // temporal average: block mean of ts consecutive post-step states
                float accE = sk[SV_ACC_E * npairs] + En;
                float accI = sk[SV_ACC_I * npairs] + In;
                if (sample_now) {
                    const float xE = accE * inv_ts, xI = accI * inv_ts;
                    if (t < a.T) {
                        a.series[t * (int64_t)N * P + (int64_t)k * P + p] = xE;
                        if (t >= a.transient) {
                            // compensated (Kahan) running sums of the samples
                            float sE = sk[SV_SUM_E * npairs], cE = sk[SV_CMP_E * npairs];
                            float y = xE - cE, tt = sE + y;
                            sk[SV_CMP_E * npairs] = (tt - sE) - y;
                            sk[SV_SUM_E * npairs] = tt;
                            float sI = sk[SV_SUM_I * npairs], cI = sk[SV_CMP_I * npairs];
                            y = xI - cI; tt = sI + y;
                            sk[SV_CMP_I * npairs] = (tt - sI) - y;
                            sk[SV_SUM_I * npairs] = tt;
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
        const int v = i / npairs, rem = i - v * npairs, k = rem / PB, qq = rem - k * PB;
        if (qq < tile.nq) a.state[((int64_t)v * N + k) * P + grp.p_base + tile.q0 + qq] = st[i];
    }
    if (active && flags) atomicOr(a.status + p, flags);
}

// ---------------------------------------------------------------------------
// Transfer function at explicit points (parity tests of the a3 step).
// ---------------------------------------------------------------------------
__global__ void tf_eval_kernel(DevModel m, int pop, int64_t n, const float* __restrict__ x_e,
                               const float* __restrict__ x_i, const float* __restrict__ W,
                               const float* __restrict__ E_L, float* __restrict__ out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        float F[6], muV;
        transfer_x(m, pop == 0 ? m.P_e : m.P_i, E_L[i], W[i], x_e[i], x_i[i], F, muV);
        for (int c = 0; c < 6; ++c) out[i * 7 + c] = F[c];
        out[i * 7 + 6] = muV;
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
    init_state_kernel<<<1024, 256, 0, s>>>(a.state, a.status, NP, a.P, a.m.E0, a.m.I0);
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

cudaError_t launch_tf_eval(const DevModel& m, int pop, int64_t n, const float* x_e, const float* x_i,
                           const float* W, const float* E_L, float* out, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    note_launch();
    tf_eval_kernel<<<(int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096), 256, 0, s>>>(
        m, pop, n, x_e, x_i, W, E_L, out);
    return cudaGetLastError();
}

}  // namespace tvbx

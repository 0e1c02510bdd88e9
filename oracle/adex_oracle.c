/*
 * FP64 CPU oracle for the TVB-AdEx parameter sweep (arXiv 2311.13337).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the slow, plain reference that the
 * CUDA engine is checked against. It shares no code, header, table or helper
 * with the engine; only tests, the smoke check and the CPU-baseline leg of the
 * benchmark may load it. Nothing on the product path may call it.
 *
 * What it computes, in the paper's order (Section 2 "Mean Field model",
 * "Transfer Function", "TVB-AdEx to GPU", "MPI" last paragraph):
 *   - Eq. 1: second-order rate equations for nu_e, nu_i;
 *   - Eq. 2: covariance equations for c_ee, c_ei, c_ii;
 *   - Eq. 3: adaptation W_e (and W_i, which is identically zero with b_i=a_i=0);
 *   - Eq. 4: Ornstein-Uhlenbeck drive noise, one process per region;
 *   - Eq. 5: transfer function F_mu(nu_e^tot + wNoise*OU + cF_mu,e,
 *            nu_i + cF_mu,i, W_mu), with nu_e^tot the delayed, weighted sum
 *            over the connectome (linear coupling, delays = length / speed);
 *   - Table 1: the second-order threshold polynomial, used as printed (mV);
 *   - forward Euler for the ODEs, Euler-Maruyama for the OU term;
 *   - the temporal-average observable (block mean of tavg_steps steps);
 *   - per-set status bits: non-finite state, E/I clamped, and "diverged" when
 *     a covariance passes C_div (the moment closure has broken down; the
 *     dynamics are not altered).
 * The transfer-function template (mu_V, sigma_V, tau_V and the normalisation
 * of the polynomial variables) is the semi-analytic one of Zerlaut et al. 2018,
 * which the paper cites for it; its derivatives with respect to the two input
 * rates are analytic (second-order forward mode, value + gradient + Hessian).
 *
 * Readings of points the paper leaves open (each also listed in the design
 * notes): the local rate nu_e of region k enters its own excitatory input; the
 * a_e term of Eq. 3 carries 1/tau_w; sigma of Eq. 4 is the noise amplitude;
 * delays are rint(length / (speed*dt)) with ties to even; the prehistory is
 * constant and equal to the initial rate; everything in a step uses the state
 * at that step, OU is advanced after use, then E and I are clamped; noise comes
 * from Philox4x32-10 (Salmon et al., SC'11) through Box-Muller.
 *
 * Pinned by the CPU tests against: the ATen Philox engine, normal-distribution
 * statistics, the closed-form OU variance and autocorrelation, Campbell's
 * theorem for sigma_V and tau_V, a root solve for mu_V, the Gaussian survival
 * function for F, Richardson finite differences for the derivatives, a
 * Lyapunov solve of Eq. 2 at the fixed point, a brute-force integrator on 2-4
 * regions, g=0 independence, zero-delay coupling and shard invariance.
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -fPIC -shared (no FMA contraction,
 * so x86_64 and aarch64 hosts produce the same bits).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ----------------------------------------------------------------------------
 * Model constants (fixed for a sweep). Units: ms, kHz, mV, nS, pF, pA.
 * -------------------------------------------------------------------------- */
typedef struct {
    double g_L, C_m, E_e, E_i, Q_e, Q_i, tau_e, tau_i;
    double K_e, K_i;            /* synaptic inputs per cell from the e / i pools */
    double N_e, N_i;            /* population sizes in the finite-size term of Eq. 2 */
    double T;                   /* time constant of Eq. 1-2 */
    double P_e[10], P_i[10];    /* Table 1, RS row for e and FS row for i (mV) */
    double mu0, dmu0, sig0, dsig0, tau0, dtau0; /* polynomial normalisation */
    double rate_floor;          /* added to K*nu so that sigma_V stays positive */
    double tau_OU, mu_OU, sigma_OU;
    double b_i, a_i, tau_w_i;   /* inhibitory adaptation (zero by default) */
    double E_min, E_max;        /* clamp of E and I after each step (kHz) */
    double E0, I0;              /* initial rates (kHz) */
    double C_div;               /* a covariance beyond this magnitude marks the set
                                   as diverged (status only; kHz^2) */
} or_model;

/* Per-set parameter vector: the sweepable axes, in this order. */
enum { OR_G, OR_B_E, OR_TAU_W_E, OR_E_L_E, OR_E_L_I, OR_SPEED, OR_A_E,
       OR_W_NOISE, OR_CF_EE, OR_CF_EI, OR_CF_IE, OR_CF_II, OR_NPRM };

/* Status bits per set. */
#define OR_ST_NONFINITE 1u
#define OR_ST_CLAMP_HI  2u
#define OR_ST_CLAMP_LO  4u
#define OR_ST_DIVERGED  16u

/* ----------------------------------------------------------------------------
 * Philox4x32-10, from the SC'11 description: 10 rounds of the 4-word S-box
 * with multipliers 0xD2511F53 / 0xCD9E8D57 and the Weyl key bumps
 * 0x9E3779B9 / 0xBB67AE85 between rounds.
 * -------------------------------------------------------------------------- */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint64_t pa = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t pb = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t y0 = (uint32_t)(pb >> 32) ^ x1 ^ k0;
        uint32_t y1 = (uint32_t)pb;
        uint32_t y2 = (uint32_t)(pa >> 32) ^ x3 ^ k1;
        uint32_t y3 = (uint32_t)pa;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Standard normal for (step n, region k, set p or 0): Box-Muller on the first
 * two Philox words, u1 = (x0 + 1) 2^-32 in (0, 1], u2 = x1 2^-32 in [0, 1). */
double or_normal(uint64_t seed, uint32_t n, uint32_t k, uint32_t p)
{
    uint32_t ctr[4] = { n, k, p, 0u };
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    uint32_t x[4];
    or_philox4x32_10(ctr, key, x);
    const double two32 = 4294967296.0;
    double u1 = ((double)x[0] + 1.0) / two32;
    double u2 = (double)x[1] / two32;
    return sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2);
}

/* Eq. 4 by Euler-Maruyama, for one region: OU[0] = 0 and
 * OU[n+1] = OU[n] + dt/tau (mu - OU[n]) + sigma sqrt(dt)/tau xi[n]. */
void or_ou_series(const or_model* m, double dt, uint64_t seed, uint32_t k, uint32_t p,
                  int64_t n_steps, double* out)
{
    double ou = 0.0;
    for (int64_t n = 0; n < n_steps; ++n) {
        out[n] = ou;
        double xi = or_normal(seed, (uint32_t)n, k, p);
        ou = ou + dt / m->tau_OU * (m->mu_OU - ou) + m->sigma_OU * sqrt(dt) / m->tau_OU * xi;
    }
}

/* ----------------------------------------------------------------------------
 * Second-order jets in the two input rates (x_e, x_i): value, gradient and
 * Hessian. Every intermediate of the transfer function is carried as a jet.
 * -------------------------------------------------------------------------- */
typedef struct { double v, e, i, ee, ei, ii; } jet;

static jet j_const(double c) { jet r = { c, 0, 0, 0, 0, 0 }; return r; }
static jet j_add(jet a, jet b)
{
    jet r = { a.v + b.v, a.e + b.e, a.i + b.i, a.ee + b.ee, a.ei + b.ei, a.ii + b.ii };
    return r;
}
static jet j_sub(jet a, jet b)
{
    jet r = { a.v - b.v, a.e - b.e, a.i - b.i, a.ee - b.ee, a.ei - b.ei, a.ii - b.ii };
    return r;
}
static jet j_scale(jet a, double s)
{
    jet r = { a.v * s, a.e * s, a.i * s, a.ee * s, a.ei * s, a.ii * s };
    return r;
}
static jet j_addc(jet a, double c) { a.v += c; return a; }
static jet j_mul(jet a, jet b)
{
    jet r;
    r.v = a.v * b.v;
    r.e = a.e * b.v + a.v * b.e;
    r.i = a.i * b.v + a.v * b.i;
    r.ee = a.ee * b.v + 2.0 * a.e * b.e + a.v * b.ee;
    r.ei = a.ei * b.v + a.e * b.i + a.i * b.e + a.v * b.ei;
    r.ii = a.ii * b.v + 2.0 * a.i * b.i + a.v * b.ii;
    return r;
}
/* f(a) given f(a.v), f'(a.v), f''(a.v). */
static jet j_chain(jet a, double f0, double f1, double f2)
{
    jet r;
    r.v = f0;
    r.e = f1 * a.e;
    r.i = f1 * a.i;
    r.ee = f1 * a.ee + f2 * a.e * a.e;
    r.ei = f1 * a.ei + f2 * a.e * a.i;
    r.ii = f1 * a.ii + f2 * a.i * a.i;
    return r;
}
static jet j_recip(jet a)
{
    double q = 1.0 / a.v;
    return j_chain(a, q, -q * q, 2.0 * q * q * q);
}
static jet j_div(jet a, jet b) { return j_mul(a, j_recip(b)); }
static jet j_sqrt(jet a)
{
    double s = sqrt(a.v);
    return j_chain(a, s, 0.5 / s, -0.25 / (s * a.v));
}
static jet j_erfc(jet a)
{
    double g = 2.0 / sqrt(M_PI) * exp(-a.v * a.v);
    return j_chain(a, erfc(a.v), -g, 2.0 * a.v * g);
}

/* Intermediates of the transfer function, exported for the tests. */
typedef struct { double muG, muV, Tm, sigV, tauV, tauVN, Vthre, arg; } or_tf_aux;

/* Transfer function of one population (Eq. 5 with the Zerlaut 2018 template
 * and the Table 1 polynomial P). x_e, x_i: total excitatory and inhibitory
 * input rates (kHz); W: adaptation current (pA); E_L: leak reversal (mV).
 * Returns the jet of F (kHz) in (x_e, x_i). */
static jet or_tf_jet(const or_model* m, const double P[10], double E_L,
                     double x_e, double x_i, double W, or_tf_aux* aux)
{
    /* synaptic input rates fe = K_e nu_e, fi = K_i nu_i (non-negative part) */
    jet fe = j_const(m->K_e * (x_e > 0.0 ? x_e : 0.0) + m->rate_floor);
    fe.e = x_e > 0.0 ? m->K_e : 0.0;
    jet fi = j_const(m->K_i * (x_i > 0.0 ? x_i : 0.0) + m->rate_floor);
    fi.i = x_i > 0.0 ? m->K_i : 0.0;

    /* mean conductances and the mean voltage of the passive membrane */
    jet muGe = j_scale(fe, m->Q_e * m->tau_e);
    jet muGi = j_scale(fi, m->Q_i * m->tau_i);
    jet muG = j_addc(j_add(muGe, muGi), m->g_L);
    jet num = j_addc(j_add(j_scale(muGe, m->E_e), j_scale(muGi, m->E_i)), m->g_L * E_L - W);
    jet muV = j_div(num, muG);
    jet Tm = j_scale(j_recip(muG), m->C_m);

    /* PSP amplitudes and the shot-noise variance and correlation time */
    jet Ue = j_scale(j_div(j_sub(j_const(m->E_e), muV), muG), m->Q_e);
    jet Ui = j_scale(j_div(j_sub(j_const(m->E_i), muV), muG), m->Q_i);
    jet Ute = j_scale(Ue, m->tau_e);
    jet Uti = j_scale(Ui, m->tau_i);
    jet Ae = j_mul(fe, j_mul(Ute, Ute));
    jet Ai = j_mul(fi, j_mul(Uti, Uti));
    jet De = j_addc(Tm, m->tau_e);
    jet Di = j_addc(Tm, m->tau_i);
    jet sV2 = j_add(j_div(Ae, j_scale(De, 2.0)), j_div(Ai, j_scale(Di, 2.0)));
    jet sV = j_sqrt(sV2);
    jet tV = j_div(j_add(Ae, Ai), j_add(j_div(Ae, De), j_div(Ai, Di)));
    jet tVN = j_scale(tV, m->g_L / m->C_m);

    /* second-order threshold polynomial in the normalised variables */
    jet V = j_scale(j_addc(muV, -m->mu0), 1.0 / m->dmu0);
    jet S = j_scale(j_addc(sV, -m->sig0), 1.0 / m->dsig0);
    jet Z = j_scale(j_addc(tVN, -m->tau0), 1.0 / m->dtau0);
    jet th = j_const(P[0]);
    th = j_add(th, j_scale(V, P[1]));
    th = j_add(th, j_scale(S, P[2]));
    th = j_add(th, j_scale(Z, P[3]));
    th = j_add(th, j_scale(j_mul(V, V), P[4]));
    th = j_add(th, j_scale(j_mul(S, S), P[5]));
    th = j_add(th, j_scale(j_mul(Z, Z), P[6]));
    th = j_add(th, j_scale(j_mul(V, S), P[7]));
    th = j_add(th, j_scale(j_mul(V, Z), P[8]));
    th = j_add(th, j_scale(j_mul(S, Z), P[9]));

    /* Gaussian membrane above the threshold, per correlation time */
    jet arg = j_div(j_sub(th, muV), j_scale(sV, sqrt(2.0)));
    jet F = j_div(j_erfc(arg), j_scale(tV, 2.0));

    if (aux) {
        aux->muG = muG.v; aux->muV = muV.v; aux->Tm = Tm.v; aux->sigV = sV.v;
        aux->tauV = tV.v; aux->tauVN = tVN.v; aux->Vthre = th.v; aux->arg = arg.v;
    }
    return F;
}

/* Exported form: out6 = {F, dF/dx_e, dF/dx_i, d2F/dx_e2, d2F/dx_e dx_i, d2F/dx_i2},
 * aux8 = {muG, muV, Tm, sigV, tauV, tauVN, Vthre, arg} (nullable). */
void or_tf_eval(const or_model* m, const double P[10], double E_L, double x_e, double x_i,
                double W, double out6[6], double* aux8)
{
    or_tf_aux a;
    jet F = or_tf_jet(m, P, E_L, x_e, x_i, W, &a);
    out6[0] = F.v; out6[1] = F.e; out6[2] = F.i; out6[3] = F.ee; out6[4] = F.ei; out6[5] = F.ii;
    if (aux8) {
        aux8[0] = a.muG; aux8[1] = a.muV; aux8[2] = a.Tm; aux8[3] = a.sigV;
        aux8[4] = a.tauV; aux8[5] = a.tauVN; aux8[6] = a.Vthre; aux8[7] = a.arg;
    }
}

/* Integer delay in steps: rint(length / (speed * dt)), ties to even (the
 * default rounding mode). length in mm, speed in m/s = mm/ms, dt in ms. */
int64_t or_delay_steps(double length_mm, double speed, double dt)
{
    return (int64_t)rint(length_mm / (speed * dt));
}

/* ----------------------------------------------------------------------------
 * One parameter set, integrated with a full (non-ring) history of E.
 * -------------------------------------------------------------------------- */
static uint32_t simulate_one(const or_model* m, int N, const double* Wc, const double* L,
                             const double* prm, double dt, int64_t S, int ts,
                             uint64_t seed, int noise_per_set, uint32_t p_global,
                             double* serE, double* serI, double* state_out)
{
    const double g = prm[OR_G], b_e = prm[OR_B_E], tau_w_e = prm[OR_TAU_W_E];
    const double E_L_e = prm[OR_E_L_E], E_L_i = prm[OR_E_L_I], speed = prm[OR_SPEED];
    const double a_e = prm[OR_A_E], w_noise = prm[OR_W_NOISE];
    const double cF_ee = prm[OR_CF_EE], cF_ei = prm[OR_CF_EI];
    const double cF_ie = prm[OR_CF_IE], cF_ii = prm[OR_CF_II];
    const int64_t T_out = S / ts;
    uint32_t status = 0;
    for (int a = 0; a < OR_NPRM; ++a)
        if (!isfinite(prm[a])) status |= OR_ST_NONFINITE;   /* a non-finite parameter */

    /* delays for this set's speed */
    int64_t* d = (int64_t*)malloc(sizeof(int64_t) * (size_t)N * (size_t)N);
    int64_t D = 0;
    for (int k = 0; k < N; ++k)
        for (int j = 0; j < N; ++j) {
            int64_t v = or_delay_steps(L[(size_t)k * N + j], speed, dt);
            if (v < 0) v = 0;
            d[(size_t)k * N + j] = v;
            if (Wc[(size_t)k * N + j] != 0.0 && v > D) D = v;
        }

    /* history: hist[j][D + m] = E_j at step m, for m in [-D, S] */
    const int64_t HL = D + S + 1;
    double* hist = (double*)malloc(sizeof(double) * (size_t)N * (size_t)HL);
    double *E = malloc(sizeof(double) * N), *I = malloc(sizeof(double) * N);
    double *Cee = malloc(sizeof(double) * N), *Cei = malloc(sizeof(double) * N);
    double *Cii = malloc(sizeof(double) * N), *We = malloc(sizeof(double) * N);
    double *Wi = malloc(sizeof(double) * N), *OU = malloc(sizeof(double) * N);
    double *c = malloc(sizeof(double) * N);
    double *accE = calloc((size_t)N, sizeof(double)), *accI = calloc((size_t)N, sizeof(double));

    for (int k = 0; k < N; ++k) {
        E[k] = m->E0; I[k] = m->I0;
        Cee[k] = Cei[k] = Cii[k] = 0.0;
        We[k] = Wi[k] = 0.0;
        OU[k] = 0.0;
        for (int64_t t = 0; t <= D; ++t) hist[(size_t)k * HL + t] = m->E0; /* constant prehistory */
    }

    const double rT = 1.0 / m->T;
    for (int64_t n = 0; n < S; ++n) {
        /* delayed linear coupling from the state history up to step n */
        for (int k = 0; k < N; ++k) {
            double s = 0.0;
            for (int j = 0; j < N; ++j) {
                double w = Wc[(size_t)k * N + j];
                if (w != 0.0) s += w * hist[(size_t)j * HL + D + n - d[(size_t)k * N + j]];
            }
            c[k] = g * s;
        }
        for (int k = 0; k < N; ++k) {
            const double Ek = E[k], Ik = I[k];
            const double ce = Cee[k], cx = Cei[k], ci = Cii[k];
            const double exc = Ek + c[k] + w_noise * OU[k];
            or_tf_aux ae, ai;
            jet Fe = or_tf_jet(m, m->P_e, E_L_e, exc + cF_ee, Ik + cF_ei, We[k], &ae);
            jet Fi = or_tf_jet(m, m->P_i, E_L_i, exc + cF_ie, Ik + cF_ii, Wi[k], &ai);

            /* Eq. 1 */
            double dE = ((Fe.v - Ek) + 0.5 * (ce * Fe.ee + 2.0 * cx * Fe.ei + ci * Fe.ii)) * rT;
            double dI = ((Fi.v - Ik) + 0.5 * (ce * Fi.ee + 2.0 * cx * Fi.ei + ci * Fi.ii)) * rT;
            /* Eq. 2 */
            double dCee = (Fe.v * (rT - Fe.v) / m->N_e + (Fe.v - Ek) * (Fe.v - Ek)
                           + 2.0 * ce * Fe.e + 2.0 * cx * Fe.i - 2.0 * ce) * rT;
            double dCei = ((Fe.v - Ek) * (Fi.v - Ik) + cx * Fe.e + ci * Fe.i + ce * Fi.e + cx * Fi.i
                           - 2.0 * cx) * rT;
            double dCii = (Fi.v * (rT - Fi.v) / m->N_i + (Fi.v - Ik) * (Fi.v - Ik)
                           + 2.0 * cx * Fi.e + 2.0 * ci * Fi.i - 2.0 * ci) * rT;
            /* Eq. 3 */
            double dWe = -We[k] / tau_w_e + b_e * Ek + a_e * (ae.muV - E_L_e) / tau_w_e;
            double dWi = -Wi[k] / m->tau_w_i + m->b_i * Ik + m->a_i * (ai.muV - E_L_i) / m->tau_w_i;

            /* forward Euler */
            double En = Ek + dt * dE, In = Ik + dt * dI;
            Cee[k] = ce + dt * dCee;
            Cei[k] = cx + dt * dCei;
            Cii[k] = ci + dt * dCii;
            if (fabs(Cee[k]) > m->C_div || fabs(Cei[k]) > m->C_div || fabs(Cii[k]) > m->C_div)
                status |= OR_ST_DIVERGED;
            We[k] = We[k] + dt * dWe;
            Wi[k] = Wi[k] + dt * dWi;

            /* Eq. 4, advanced after use */
            double xi = or_normal(seed, (uint32_t)n, (uint32_t)k, noise_per_set ? p_global : 0u);
            OU[k] = OU[k] + dt / m->tau_OU * (m->mu_OU - OU[k]) + m->sigma_OU * sqrt(dt) / m->tau_OU * xi;

            if (!isfinite(En) || !isfinite(In)) status |= OR_ST_NONFINITE;
            if (En > m->E_max) { En = m->E_max; status |= OR_ST_CLAMP_HI; }
            if (En < m->E_min) { En = m->E_min; status |= OR_ST_CLAMP_LO; }
            if (In > m->E_max) { In = m->E_max; status |= OR_ST_CLAMP_HI; }
            if (In < m->E_min) { In = m->E_min; status |= OR_ST_CLAMP_LO; }
            E[k] = En; I[k] = In;
            hist[(size_t)k * HL + D + n + 1] = En;

            /* temporal average: block mean of ts consecutive post-step states */
            accE[k] += En; accI[k] += In;
        }
        if ((n + 1) % ts == 0) {
            int64_t t = (n + 1) / ts - 1;
            if (t < T_out)
                for (int k = 0; k < N; ++k) {
                    if (serE) serE[(size_t)k * T_out + t] = accE[k] / ts;
                    if (serI) serI[(size_t)k * T_out + t] = accI[k] / ts;
                    accE[k] = 0.0; accI[k] = 0.0;
                }
        }
    }
    if (state_out)
        for (int k = 0; k < N; ++k) {
            state_out[0 * N + k] = E[k];  state_out[1 * N + k] = I[k];
            state_out[2 * N + k] = Cee[k]; state_out[3 * N + k] = Cei[k];
            state_out[4 * N + k] = Cii[k]; state_out[5 * N + k] = We[k];
            state_out[6 * N + k] = Wi[k];  state_out[7 * N + k] = OU[k];
        }
    for (int k = 0; k < N; ++k)
        if (!isfinite(Cee[k]) || !isfinite(Cei[k]) || !isfinite(Cii[k]) || !isfinite(We[k]))
            status |= OR_ST_NONFINITE;

    free(d); free(hist); free(E); free(I); free(Cee); free(Cei); free(Cii);
    free(We); free(Wi); free(OU); free(c); free(accE); free(accI);
    return status;
}

/* Sweep: P sets, each with its own parameter vector prm[p*OR_NPRM + axis].
 * W, L: N x N row-major connectome weights u_kj and tract lengths (mm).
 * Outputs (each nullable): serE/serI [P][N][S/ts] tavg series (kHz),
 * state_out [P][8][N] final state, status [P]. p_offset is the global index of
 * set 0 (it keys per-set noise). n_threads <= 0 uses the OpenMP default. */
int or_simulate(const or_model* m, int N, const double* W, const double* L, int P,
                const double* prm, double dt, int64_t S, int ts, uint64_t seed,
                int noise_per_set, int64_t p_offset, int n_threads,
                double* serE, double* serI, double* state_out, uint32_t* status)
{
    if (N <= 0 || P < 0 || S < 0 || ts <= 0 || dt <= 0.0) return -1;
    const int64_t T_out = S / ts;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int p = 0; p < P; ++p) {
        uint32_t st = simulate_one(m, N, W, L, prm + (size_t)p * OR_NPRM, dt, S, ts, seed,
                                   noise_per_set, (uint32_t)(p_offset + p),
                                   serE ? serE + (size_t)p * N * T_out : NULL,
                                   serI ? serI + (size_t)p * N * T_out : NULL,
                                   state_out ? state_out + (size_t)p * 8 * N : NULL);
        if (status) status[p] = st;
    }
    return 0;
}

int or_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

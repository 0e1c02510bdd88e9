// Refit of the transfer-function polynomial from single-cell simulations
// (arXiv 2311.13337, Sec. "Transfer Function": the effective threshold of the
// semi-analytic template is a second-order polynomial in the normalised
// mu_V, sigma_V, tau_V^N, Table 1, fitted to simulations of single AdEx
// neurons, Zerlaut et al. 2018).
//
// tvbx_cell_rates: one thread per cell integrates an adaptive exponential
// integrate-and-fire neuron (Brette and Gerstner 2005) driven by Poisson
// excitatory and inhibitory spike trains through exponential conductances,
// forward Euler. Each step draws the input counts from words 0 and 1 of
// Philox4x32-10 (counter (step, cell, 0, 0), key = seed) by comparison with
// integer thresholds floor(P(N <= k) 2^32) computed on the host in FP64, so
// the counts are exact integers independent of device rounding.
//
// tvbx_tf_fit: for every point with a rate in (0, 1 / (2 tau_V)), the
// template's mu_V, sigma_V, tau_V (FP64, host) and the effective threshold
// mu_V + sqrt(2) sigma_V erfcinv(2 tau_V F); the ten Table 1 coefficients
// by linear least squares (Householder QR).

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <cmath>
#include <vector>

#include "internal.h"
#include "model_device.cuh"
#include "tvbx.h"

namespace tvbx {
namespace {

constexpr int CELL_KT = 32;   // Poisson thresholds per count table (counts 0..31)

struct CellDev {
    float inv_C, gL, EL, VT, Delta, inv_Delta, Vreset, Vcut, Qe, Qi, de, di, Ee, Ei, dt;
    int32_t ref_steps;
};

__global__ void adex_cells_kernel(CellDev c, int64_t n, int32_t n_cells, const uint32_t* __restrict__ Te,
                                  const uint32_t* __restrict__ Ti, const float* __restrict__ W, int64_t n_steps,
                                  int64_t n_tr, uint64_t seed, int32_t* __restrict__ count_out)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t p = i / n_cells;
    const uint32_t* te = Te + p * CELL_KT;
    const uint32_t* ti = Ti + p * CELL_KT;
    const float w = W[p];
    float V = c.EL, ge = 0.0f, gi = 0.0f;
    int ref = 0, cnt = 0;
    for (int64_t s = 0; s < n_steps; ++s) {
        const uint4 x = philox4x32_10(make_uint4((uint32_t)s, (uint32_t)i, 0u, 0u), (uint32_t)seed,
                                      (uint32_t)(seed >> 32));
        int ne = 0, ni = 0;
        while (ne < CELL_KT && __ldg(te + ne) <= x.x) ++ne;
        while (ni < CELL_KT && __ldg(ti + ni) <= x.y) ++ni;
        ge = fmaf(ge, c.de, c.Qe * (float)ne);
        gi = fmaf(gi, c.di, c.Qi * (float)ni);
        if (ref == 0) {
            const float dV = (c.gL * (c.EL - V) + c.gL * c.Delta * expf((V - c.VT) * c.inv_Delta) + ge * (c.Ee - V) +
                              gi * (c.Ei - V) - w) * c.inv_C;
            V = fmaf(c.dt, dV, V);
            if (V >= c.Vcut) {
                V = c.Vreset;
                ref = c.ref_steps;
                if (s >= n_tr) ++cnt;
            }
        } else {
            V = c.Vreset;
            --ref;
        }
    }
    count_out[i] = cnt;
}

void poisson_thresholds(double mean, uint32_t* out)
{
    double p = std::exp(-mean), cdf = p;
    for (int k = 0; k < CELL_KT; ++k) {
        const double v = std::floor(cdf * 4294967296.0);
        out[k] = v >= 4294967295.0 ? 4294967295u : (uint32_t)v;
        p = p * mean / (double)(k + 1);
        cdf = cdf + p;
    }
}

// Inverse complementary error function: bisection, then Newton steps on erfc.
double inv_erfc(double y)
{
    double lo = -10.0, hi = 10.0;
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (std::erfc(mid) > y) lo = mid;
        else hi = mid;
    }
    double x = 0.5 * (lo + hi);
    for (int it = 0; it < 3; ++it) x -= (std::erfc(x) - y) / (-2.0 / std::sqrt(M_PI) * std::exp(-x * x));
    return x;
}

// Least squares min |A x - b| for A [m][n] (row-major, m >= n) by Householder QR.
bool least_squares(std::vector<double> A, std::vector<double> b, int m, int n, double* x)
{
    for (int k = 0; k < n; ++k) {
        double nrm = 0.0;
        for (int i = k; i < m; ++i) nrm += A[i * n + k] * A[i * n + k];
        nrm = std::sqrt(nrm);
        if (nrm == 0.0) return false;
        const double alpha = A[k * n + k] > 0 ? -nrm : nrm;
        std::vector<double> v(m - k);
        for (int i = k; i < m; ++i) v[i - k] = A[i * n + k];
        v[0] -= alpha;
        double vv = 0.0;
        for (double t : v) vv += t * t;
        if (vv == 0.0) continue;
        for (int j = k; j < n; ++j) {
            double d = 0.0;
            for (int i = k; i < m; ++i) d += v[i - k] * A[i * n + j];
            const double f = 2.0 * d / vv;
            for (int i = k; i < m; ++i) A[i * n + j] -= f * v[i - k];
        }
        double d = 0.0;
        for (int i = k; i < m; ++i) d += v[i - k] * b[i];
        const double f = 2.0 * d / vv;
        for (int i = k; i < m; ++i) b[i] -= f * v[i - k];
    }
    for (int k = n - 1; k >= 0; --k) {
        double s = b[k];
        for (int j = k + 1; j < n; ++j) s -= A[k * n + j] * x[j];
        if (A[k * n + k] == 0.0) return false;
        x[k] = s / A[k * n + k];
    }
    return true;
}

}  // namespace
}  // namespace tvbx

using namespace tvbx;

extern "C" tvbx_status tvbx_cell_defaults(int32_t pop, tvbx_cell_params* out)
{
    if (!out || (pop != 0 && pop != 1)) return report_error(TVBX_E_INVALID_ARG, "need out and pop 0 (RS) or 1 (FS)");
    out->C = 200.0;
    out->gL = 10.0;
    out->EL = -64.0;
    out->VT = -50.0;
    out->Delta = pop == 0 ? 2.0 : 0.5;
    out->Vreset = -65.0;
    out->t_ref = 5.0;
    out->Qe = 1.5;
    out->Qi = 5.0;
    out->tau_e = 5.0;
    out->tau_i = 5.0;
    out->Ee = 0.0;
    out->Ei = -80.0;
    out->Ke = 400.0;
    out->Ki = 100.0;
    return TVBX_OK;
}

extern "C" tvbx_status tvbx_cell_rates(const tvbx_cell_params* cell, int64_t n_points, const double* nu_e_khz,
                                       const double* nu_i_khz, const double* W_pA, int32_t n_cells, double T_ms,
                                       double transient_ms, double dt_ms, uint64_t seed, double* rate_khz_out)
{
    if (!cell || !nu_e_khz || !nu_i_khz || !W_pA || !rate_khz_out)
        return report_error(TVBX_E_INVALID_ARG, "NULL argument");
    if (n_points < 1 || n_cells < 1 || n_points * (int64_t)n_cells > ((int64_t)1 << 31) - 1)
        return report_error(TVBX_E_INVALID_ARG, "need n_points >= 1, n_cells >= 1, n_points n_cells < 2^31");
    if (!(dt_ms > 0.0) || !(T_ms > transient_ms) || transient_ms < 0.0 || !(cell->Delta > 0.0) || !(cell->C > 0.0))
        return report_error(TVBX_E_INVALID_ARG, "need dt_ms > 0, 0 <= transient_ms < T_ms, Delta > 0, C > 0");
    for (int64_t p = 0; p < n_points; ++p)
        if (!(nu_e_khz[p] >= 0.0) || !(nu_i_khz[p] >= 0.0) || !std::isfinite(W_pA[p]))
            return report_error(TVBX_E_INVALID_ARG, "point %lld: rates must be >= 0 and W finite", (long long)p);
    const int64_t n = n_points * n_cells;
    std::vector<uint32_t> Te(n_points * CELL_KT), Ti(n_points * CELL_KT);
    std::vector<float> W(n_points);
    for (int64_t p = 0; p < n_points; ++p) {
        poisson_thresholds(cell->Ke * nu_e_khz[p] * dt_ms, Te.data() + p * CELL_KT);
        poisson_thresholds(cell->Ki * nu_i_khz[p] * dt_ms, Ti.data() + p * CELL_KT);
        W[p] = (float)W_pA[p];
    }
    CellDev c;
    c.inv_C = (float)(1.0 / cell->C);
    c.gL = (float)cell->gL;
    c.EL = (float)cell->EL;
    c.VT = (float)cell->VT;
    c.Delta = (float)cell->Delta;
    c.inv_Delta = (float)(1.0 / cell->Delta);
    c.Vreset = (float)cell->Vreset;
    c.Vcut = (float)(cell->VT + 5.0 * cell->Delta);
    c.Qe = (float)cell->Qe;
    c.Qi = (float)cell->Qi;
    c.de = (float)(1.0 - dt_ms / cell->tau_e);
    c.di = (float)(1.0 - dt_ms / cell->tau_i);
    c.Ee = (float)cell->Ee;
    c.Ei = (float)cell->Ei;
    c.dt = (float)dt_ms;
    c.ref_steps = (int32_t)std::lround(cell->t_ref / dt_ms);
    const int64_t n_steps = std::llround(T_ms / dt_ms), n_tr = std::llround(transient_ms / dt_ms);
    uint32_t *dTe = nullptr, *dTi = nullptr;
    float* dW = nullptr;
    int32_t* dC = nullptr;
    cudaError_t e = cudaMalloc(&dTe, sizeof(uint32_t) * Te.size());
    if (e == cudaSuccess) e = cudaMalloc(&dTi, sizeof(uint32_t) * Ti.size());
    if (e == cudaSuccess) e = cudaMalloc(&dW, sizeof(float) * W.size());
    if (e == cudaSuccess) e = cudaMalloc(&dC, sizeof(int32_t) * n);
    if (e == cudaSuccess) e = cudaMemcpy(dTe, Te.data(), sizeof(uint32_t) * Te.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dTi, Ti.data(), sizeof(uint32_t) * Ti.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dW, W.data(), sizeof(float) * W.size(), cudaMemcpyHostToDevice);
    std::vector<int32_t> counts(n);
    if (e == cudaSuccess) {
        note_launch();
        adex_cells_kernel<<<(unsigned)((n + 127) / 128), 128>>>(c, n, n_cells, dTe, dTi, dW, n_steps, n_tr, seed, dC);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(counts.data(), dC, sizeof(int32_t) * n, cudaMemcpyDeviceToHost);
    cudaFree(dTe);
    cudaFree(dTi);
    cudaFree(dW);
    cudaFree(dC);
    if (e == cudaErrorMemoryAllocation) return report_error(TVBX_E_OOM, "cell rates: out of memory");
    if (e != cudaSuccess) return report_error(TVBX_E_CUDA, "cell rates: %s", cudaGetErrorString(e));
    const double T_count = (double)(n_steps - n_tr) * dt_ms;
    for (int64_t p = 0; p < n_points; ++p) {
        int64_t s = 0;
        for (int32_t k = 0; k < n_cells; ++k) s += counts[p * n_cells + k];
        rate_khz_out[p] = (double)s / ((double)n_cells * T_count);
    }
    return TVBX_OK;
}

// Template moments of one point (the same template as the engine's transfer
// function, FP64): mu_V, sigma_V, tau_V and the normalised tau_V^N; false if
// sigma_V is not finite.
static bool tf_moments(const tvbx_model* m, double nu_e, double nu_i, double W, double EL, double* muV_o,
                       double* sigV_o,
                       double* tauV_o, double* tauVN_o)
{
    const double fe = m->K_e * std::max(nu_e, 0.0) + m->rate_floor;
    const double fi = m->K_i * std::max(nu_i, 0.0) + m->rate_floor;
    const double mGe = m->Q_e * m->tau_e * fe, mGi = m->Q_i * m->tau_i * fi;
    const double muG = m->g_L + mGe + mGi;
    const double muV = (mGe * m->E_e + mGi * m->E_i + m->g_L * EL - W) / muG;
    const double Tm = m->C_m / muG;
    const double Ue = m->Q_e * (m->E_e - muV) / muG, Ui = m->Q_i * (m->E_i - muV) / muG;
    const double Ae = fe * (Ue * m->tau_e) * (Ue * m->tau_e), Ai = fi * (Ui * m->tau_i) * (Ui * m->tau_i);
    const double s2 = Ae / (m->tau_e + Tm) + Ai / (m->tau_i + Tm);   // 2 sigma_V^2
    const double sigV = std::sqrt(0.5 * s2);
    const double tauV = (Ae + Ai) / s2;
    *muV_o = muV;
    *sigV_o = sigV;
    *tauV_o = tauV;
    *tauVN_o = tauV * m->g_L / m->C_m;
    return std::isfinite(sigV) && sigV > 0.0 && std::isfinite(tauV) && tauV > 0.0;
}

// The ten Table 1 basis functions of a point's normalised moments.
static void tf_basis(const tvbx_model* m, double muV, double sigV, double tauVN, double row[10])
{
    const double V = (muV - m->mu0) / m->dmu0, S = (sigV - m->sig0) / m->dsig0, Z = (tauVN - m->tau0) / m->dtau0;
    const double r[10] = {1.0, V, S, Z, V * V, S * S, Z * Z, V * S, V * Z, S * Z};
    for (int i = 0; i < 10; ++i) row[i] = r[i];
}

extern "C" tvbx_status tvbx_tf_fit(const tvbx_model* m, int64_t n_points, const double* nu_e_khz,
                                   const double* nu_i_khz, const double* W_pA, const double* E_L,
                                   const double* rate_khz, double P_out[10], int32_t* n_used)
{
    if (!m || !nu_e_khz || !nu_i_khz || !W_pA || !E_L || !rate_khz || !P_out)
        return report_error(TVBX_E_INVALID_ARG, "NULL argument");
    if (n_points < 1) return report_error(TVBX_E_INVALID_ARG, "need n_points >= 1");
    std::vector<double> A, b;
    int rows = 0;
    for (int64_t p = 0; p < n_points; ++p) {
        double muV, sigV, tauV, tauVN;
        const bool ok = tf_moments(m, nu_e_khz[p], nu_i_khz[p], W_pA[p], E_L[p], &muV, &sigV, &tauV, &tauVN);
        const double F = rate_khz[p];
        if (!(F > 0.0) || !(2.0 * tauV * F < 1.0) || !ok) continue;
        const double vth = muV + std::sqrt(2.0) * sigV * inv_erfc(2.0 * tauV * F);
        double row[10];
        tf_basis(m, muV, sigV, tauVN, row);
        A.insert(A.end(), row, row + 10);
        b.push_back(vth);
        ++rows;
    }
    if (n_used) *n_used = rows;
    if (rows < 10) return report_error(TVBX_E_NUMERIC, "only %d points with a rate in (0, 1 / (2 tau_V))", rows);
    if (!least_squares(A, b, rows, 10, P_out)) return report_error(TVBX_E_NUMERIC, "rank-deficient fit");
    return TVBX_OK;
}

// Second stage of the fit: the coefficients that minimise the squared error
// of the template's rate F(P) = erfc((V_thre(P) - mu_V) / (sqrt(2) sigma_V)) /
// (2 tau_V), V_thre(P) = sum_i P_i B_i, over every point with a finite rate
// (silent and saturated points included). Levenberg-Marquardt from P_init
// with the analytic Jacobian dF/dP_i = -exp(-z^2) B_i / (sqrt(2 pi) sigma_V
// tau_V); each step solves the damped system [J; sqrt(lambda) D] d = [-r; 0]
// (D = the column norms of J) by Householder QR.
extern "C" tvbx_status tvbx_tf_refit(const tvbx_model* m, int64_t n_points, const double* nu_e_khz,
                                     const double* nu_i_khz, const double* W_pA, const double* E_L,
                                     const double* rate_khz, const double P_init[10], int32_t max_iter,
                                     double P_out[10], double* rms_out, int32_t* n_used)
{
    if (!m || !nu_e_khz || !nu_i_khz || !W_pA || !E_L || !rate_khz || !P_init || !P_out)
        return report_error(TVBX_E_INVALID_ARG, "NULL argument");
    if (n_points < 1 || max_iter < 0) return report_error(TVBX_E_INVALID_ARG, "need n_points >= 1 and max_iter >= 0");
    struct Pt { double muV, sigV, tauV, B[10], F; };
    std::vector<Pt> pts;
    for (int64_t p = 0; p < n_points; ++p) {
        Pt q;
        double tauVN;
        if (!std::isfinite(rate_khz[p]) || rate_khz[p] < 0.0) continue;
        if (!tf_moments(m, nu_e_khz[p], nu_i_khz[p], W_pA[p], E_L[p], &q.muV, &q.sigV, &q.tauV, &tauVN)) continue;
        tf_basis(m, q.muV, q.sigV, tauVN, q.B);
        q.F = rate_khz[p];
        pts.push_back(q);
    }
    const int n = (int)pts.size();
    if (n_used) *n_used = n;
    if (n < 10) return report_error(TVBX_E_NUMERIC, "only %d points with a finite rate", n);
    const double c_erf = 1.0 / std::sqrt(2.0 * M_PI);
    auto residuals = [&](const double* P, std::vector<double>& r, std::vector<double>* J) {
        double cost = 0.0;
        for (int p = 0; p < n; ++p) {
            const Pt& q = pts[p];
            double vth = 0.0;
            for (int i = 0; i < 10; ++i) vth += P[i] * q.B[i];
            const double z = (vth - q.muV) / (std::sqrt(2.0) * q.sigV);
            r[p] = std::erfc(z) / (2.0 * q.tauV) - q.F;
            cost += r[p] * r[p];
            if (J) {
                const double g = -c_erf * std::exp(-z * z) / (q.sigV * q.tauV);
                for (int i = 0; i < 10; ++i) (*J)[(size_t)p * 10 + i] = g * q.B[i];
            }
        }
        return cost;
    };
    double P[10], Pn[10];
    for (int i = 0; i < 10; ++i) P[i] = P_init[i];
    std::vector<double> r(n), rn(n), J((size_t)n * 10);
    double cost = residuals(P, r, &J);
    if (!std::isfinite(cost)) return report_error(TVBX_E_NUMERIC, "the rates at P_init are not finite");
    double lambda = 1e-3;
    std::vector<double> Aug((size_t)(n + 10) * 10), rhs(n + 10);
    for (int it = 0; it < max_iter; ++it) {
        double D[10];
        for (int i = 0; i < 10; ++i) {
            double s = 0.0;
            for (int p = 0; p < n; ++p) s += J[(size_t)p * 10 + i] * J[(size_t)p * 10 + i];
            D[i] = std::sqrt(s) > 0.0 ? std::sqrt(s) : 1.0;
        }
        bool accepted = false;
        while (!accepted && lambda < 1e16) {
            std::copy(J.begin(), J.end(), Aug.begin());
            for (int p = 0; p < n; ++p) rhs[p] = -r[p];
            for (int i = 0; i < 10; ++i) {
                for (int j = 0; j < 10; ++j) Aug[(size_t)(n + i) * 10 + j] = i == j ? std::sqrt(lambda) * D[i] : 0.0;
                rhs[n + i] = 0.0;
            }
            double d[10];
            if (!least_squares(Aug, rhs, n + 10, 10, d)) return report_error(TVBX_E_NUMERIC, "singular step");
            for (int i = 0; i < 10; ++i) Pn[i] = P[i] + d[i];
            const double cn = residuals(Pn, rn, nullptr);
            if (std::isfinite(cn) && cn < cost) {
                const double gain = cost - cn;
                for (int i = 0; i < 10; ++i) P[i] = Pn[i];
                cost = residuals(P, r, &J);
                lambda = std::max(lambda * 0.3, 1e-12);
                accepted = true;
                if (gain <= 1e-15 * cost) it = max_iter;   // converged
            } else {
                lambda *= 10.0;
            }
        }
        if (!accepted) break;   // no descent at any damping: a minimum
    }
    for (int i = 0; i < 10; ++i) P_out[i] = P[i];
    if (rms_out) *rms_out = std::sqrt(cost / n);
    return TVBX_OK;
}

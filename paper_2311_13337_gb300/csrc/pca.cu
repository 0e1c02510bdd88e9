// Principal components of the per-set FC matrices: the 20 FC coefficients
// the surrogate network predicts. The paper analyses FC (Sec. "Output",
// Eq. 6); reducing each set's FC to a few coefficients is this library's
// choice of surrogate target.
//
// For P sets of N regions: V[p] = upper triangle (k < j, row by row) of FC_p,
// M = N (N - 1) / 2 entries; mu = mean of the rows; C = (V - mu)^T (V - mu)
// (M x M, FP32 SIMT product). The leading eigenvectors of C come from
// subspace iteration with k' = n_comp + 12 columns: Z = C Q, Q = Z R^{-1}
// with R the Cholesky factor of Z^T Z, column-scaled (done twice per step:
// CholeskyQR2);
// then Rayleigh-Ritz: H = Q^T C Q, whose eigenpairs (cyclic Jacobi, FP64, on
// the host: k' x k') give the components U = Q E. Eigenvalues are reported
// per set (divided by P); each component's largest-magnitude entry is made
// positive. Coefficients: (V - mu) U^T.

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "gemm_simt.cuh"
#include "internal.h"
#include "model_device.cuh"
#include "tvbx.h"

namespace tvbx {
namespace {

__global__ void pca_triu_kernel(const float* __restrict__ fc, int N, int64_t P, const int2* __restrict__ kj, int M,
                                float* __restrict__ V)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= P * M) return;
    const int64_t p = i / M;
    const int e = (int)(i - p * M);
    const int2 q = kj[e];
    V[i] = fc[(p * N + q.x) * N + q.y];
}

// Column means (FP64 sums) and centring in place; grid = ceil(M / 32).
__global__ void pca_center_kernel(float* __restrict__ V, int64_t P, int M, float* __restrict__ mu)
{
    const int e = blockIdx.x * 32 + (threadIdx.x & 31);
    const int q = threadIdx.x >> 5;   // 8 row groups
    double s = 0.0;
    if (e < M)
        for (int64_t p = q; p < P; p += 8) s += V[p * M + e];
    __shared__ double red[8][33];
    red[q][threadIdx.x & 31] = s;
    __syncthreads();
    __shared__ float m_sh[32];
    if (q == 0) {
        double t = 0.0;
        for (int i = 0; i < 8; ++i) t += red[i][threadIdx.x & 31];
        m_sh[threadIdx.x] = (float)(t / (double)P);
        if (e < M) mu[e] = m_sh[threadIdx.x];
    }
    __syncthreads();
    if (e < M) {
        const float m = m_sh[threadIdx.x & 31];
        for (int64_t p = q; p < P; p += 8) V[p * M + e] -= m;
    }
}

__global__ void pca_subtract_kernel(float* __restrict__ V, int64_t P, int M, const float* __restrict__ mu)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= P * M) return;
    V[i] -= mu[i % M];
}

// G[i][j] = sum_m A[m][i] B[m][j] (A, B: [M][k]) with FP64 accumulation; one
// block per (i, j).
__global__ void pca_gram_kernel(const float* __restrict__ A, const float* __restrict__ B, int M, int k,
                                double* __restrict__ G)
{
    const int i = blockIdx.x, j = blockIdx.y;
    double s = 0.0;
    for (int m = threadIdx.x; m < M; m += blockDim.x) s += (double)A[(int64_t)m * k + i] * (double)B[(int64_t)m * k + j];
    __shared__ double red[256];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) G[i * k + j] = red[0];
}

__global__ void pca_random_kernel(float* __restrict__ Q, int64_t n, uint64_t seed)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint4 r = philox4x32_10(make_uint4((uint32_t)i, (uint32_t)(i >> 32), 0x9CAu, 0u), (uint32_t)seed,
                                  (uint32_t)(seed >> 32));
    Q[i] = ((float)r.x + 0.5f) * 2.3283064365386963e-10f - 0.5f;
}

// Cyclic Jacobi eigen-decomposition of the symmetric n x n matrix A (row
// major, destroyed); eigenvalues w, eigenvectors in the columns of E.
void jacobi_eigen(std::vector<double>& A, int n, std::vector<double>& w, std::vector<double>& E)
{
    E.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) E[(size_t)i * n + i] = 1.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = i + 1; j < n; ++j) off += A[(size_t)i * n + j] * A[(size_t)i * n + j];
        if (off < 1e-30) break;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                const double apq = A[(size_t)p * n + q];
                if (fabs(apq) < 1e-300) continue;
                const double app = A[(size_t)p * n + p], aqq = A[(size_t)q * n + q];
                const double theta = (aqq - app) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {   // A <- J^T A J
                    const double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
                    A[(size_t)k * n + p] = c * akp - s * akq;
                    A[(size_t)k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {
                    const double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
                    A[(size_t)p * n + k] = c * apk - s * aqk;
                    A[(size_t)q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    const double ekp = E[(size_t)k * n + p], ekq = E[(size_t)k * n + q];
                    E[(size_t)k * n + p] = c * ekp - s * ekq;
                    E[(size_t)k * n + q] = s * ekp + c * ekq;
                }
            }
    }
    w.resize(n);
    for (int i = 0; i < n; ++i) w[i] = A[(size_t)i * n + i];
}

// Inverse of the upper Cholesky factor R of the SPD matrix G = Z^T Z (k x k,
// FP64): G = R^T R. The factorisation runs on the column-scaled G' = D^-1 G
// D^-1, D = sqrt(diag G) (the columns of Z = C Q have norms of the order of
// the eigenvalues and are nearly orthogonal, so G' is well conditioned where
// G is not), and R = R' D. Returns false if a column is (numerically) zero or
// G' is not positive definite.
bool chol_inv_upper(const std::vector<double>& G0, int k, std::vector<double>& Rinv)
{
    std::vector<double> D(k), G((size_t)k * k);
    double dmax = 0.0;
    for (int j = 0; j < k; ++j) dmax = std::max(dmax, G0[(size_t)j * k + j]);
    for (int j = 0; j < k; ++j) {
        const double d = G0[(size_t)j * k + j];
        if (!(d > 1e-24 * dmax) || !(dmax > 0.0)) return false;
        D[j] = sqrt(d);
    }
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < k; ++j) G[(size_t)i * k + j] = G0[(size_t)i * k + j] / (D[i] * D[j]);
    std::vector<double> R((size_t)k * k, 0.0);
    for (int j = 0; j < k; ++j) {
        double s = G[(size_t)j * k + j];
        for (int i = 0; i < j; ++i) s -= R[(size_t)i * k + j] * R[(size_t)i * k + j];
        if (!(s > 0.0)) return false;
        R[(size_t)j * k + j] = sqrt(s);
        for (int c = j + 1; c < k; ++c) {
            double t = G[(size_t)j * k + c];
            for (int i = 0; i < j; ++i) t -= R[(size_t)i * k + j] * R[(size_t)i * k + c];
            R[(size_t)j * k + c] = t / R[(size_t)j * k + j];
        }
    }
    Rinv.assign((size_t)k * k, 0.0);
    for (int j = k - 1; j >= 0; --j) {   // back substitution: R Rinv = I
        Rinv[(size_t)j * k + j] = 1.0 / R[(size_t)j * k + j];
        for (int c = j + 1; c < k; ++c) {
            double t = 0.0;
            for (int i = j + 1; i <= c; ++i) t += R[(size_t)j * k + i] * Rinv[(size_t)i * k + c];
            Rinv[(size_t)j * k + c] = -t / R[(size_t)j * k + j];
        }
    }
    for (int a = 0; a < k; ++a)   // (R' D)^-1 = D^-1 R'^-1
        for (int c = 0; c < k; ++c) Rinv[(size_t)a * k + c] /= D[a];
    return true;
}

std::vector<int2> triu_pairs(int N)
{
    std::vector<int2> kj;
    for (int k = 0; k < N; ++k)
        for (int j = k + 1; j < N; ++j) kj.push_back(make_int2(k, j));
    return kj;
}

struct DevMem {
    std::vector<void*> ptrs;
    cudaStream_t s;
    explicit DevMem(cudaStream_t st) : s(st) {}
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
    ~DevMem()
    {
        for (void* q : ptrs) cudaFreeAsync(q, s);
    }
};

#define PCK(call, what)                                                                              \
    do {                                                                                             \
        cudaError_t e_ = (call);                                                                     \
        if (e_ == cudaErrorMemoryAllocation) return report_error(TVBX_E_OOM, "%s: out of memory", what); \
        if (e_ != cudaSuccess) return report_error(TVBX_E_CUDA, "%s: %s", what, cudaGetErrorString(e_)); \
    } while (0)

// Y (k x k, host FP64) = A^T B for device A, B [M][k], accumulated in FP64
// (the columns of C Q can be nearly parallel; FP32 sums would make A^T A
// indefinite).
tvbx_status small_product(const float* A, const float* B, int M, int k, double* dtmp, std::vector<double>& out,
                          cudaStream_t s)
{
    note_launch();
    pca_gram_kernel<<<dim3(k, k), 256, 0, s>>>(A, B, M, k, dtmp);
    PCK(cudaGetLastError(), "PCA product");
    out.resize((size_t)k * k);
    PCK(cudaMemcpyAsync(out.data(), dtmp, sizeof(double) * k * k, cudaMemcpyDeviceToHost, s), "PCA product");
    PCK(cudaStreamSynchronize(s), "PCA product");
    return TVBX_OK;
}

// Q = Z S for device Z [M][k] and host S (k x k): C(m = i, n = c) = sum_a Z[i][a] S[a][c].
tvbx_status right_multiply(const float* Z, int M, int k, const std::vector<double>& S, int kout, float* dS, float* Q,
                           cudaStream_t s)
{
    std::vector<float> h((size_t)k * kout);
    for (int a = 0; a < k; ++a)
        for (int c = 0; c < kout; ++c) h[(size_t)a * kout + c] = (float)S[(size_t)a * k + c];
    PCK(cudaMemcpyAsync(dS, h.data(), sizeof(float) * h.size(), cudaMemcpyHostToDevice, s), "PCA small copy");
    GemmArgs g{};
    g.A = Z; g.sam = k; g.sak = 1;
    g.B = dS; g.sbn = 1; g.sbk = kout;
    g.C = Q; g.ldc = kout;
    g.M = M; g.N = kout; g.K = k;
    PCK((gemm<float, float, EPI_STORE>(g, 1, s)), "PCA right product");
    PCK(cudaStreamSynchronize(s), "PCA right product");   // h and dS are reused
    return TVBX_OK;
}

}  // namespace
}  // namespace tvbx

using namespace tvbx;

extern "C" tvbx_status tvbx_fc_pca(const float* fc, int32_t n_regions, int64_t n_sets, int32_t n_comp, int32_t n_iter,
                                   float* mean_out, float* comps_out, float* coef_out, float* eigvals_out,
                                   void* cuda_stream)
{
    const int N = n_regions;
    const int64_t P = n_sets;
    if (!fc || !mean_out || !comps_out) return report_error(TVBX_E_INVALID_ARG, "NULL fc, mean_out or comps_out");
    if (N < 3 || N > 512 || P < 2 || P > (1ll << 31) - 1) return report_error(TVBX_E_INVALID_ARG, "need 3 <= n_regions <= 512, n_sets >= 2");
    const int M = N * (N - 1) / 2;
    if (n_comp < 1 || n_comp > 64 || n_comp > M || n_iter < 1 || n_iter > 1000)
        return report_error(TVBX_E_INVALID_ARG, "need 1 <= n_comp <= min(64, N(N-1)/2) and 1 <= n_iter <= 1000");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int kp = std::min(M, n_comp + 12);
    DevMem mem(s);
    float *V, *C, *Q, *Z, *dS;
    double* dtmp;
    int2* kj;
    PCK(mem.get(&V, (size_t)P * M), "PCA rows");
    PCK(mem.get(&C, (size_t)M * M), "PCA covariance");
    PCK(mem.get(&Q, (size_t)M * kp), "PCA basis");
    PCK(mem.get(&Z, (size_t)M * kp), "PCA basis");
    PCK(mem.get(&dS, (size_t)kp * kp), "PCA small");
    PCK(mem.get(&dtmp, (size_t)kp * kp), "PCA small");
    PCK(mem.get(&kj, (size_t)M), "PCA index");
    const std::vector<int2> pairs = triu_pairs(N);
    PCK(cudaMemcpyAsync(kj, pairs.data(), sizeof(int2) * M, cudaMemcpyHostToDevice, s), "PCA index");
    note_launch();
    pca_triu_kernel<<<(unsigned)((P * M + 255) / 256), 256, 0, s>>>(fc, N, P, kj, M, V);
    PCK(cudaGetLastError(), "PCA rows");
    note_launch();
    pca_center_kernel<<<(M + 31) / 32, 256, 0, s>>>(V, P, M, mean_out);
    PCK(cudaGetLastError(), "PCA centre");
    {   // C = V^T V
        GemmArgs g{};
        g.A = V; g.sam = 1; g.sak = M;
        g.B = V; g.sbn = 1; g.sbk = M;
        g.C = C; g.ldc = M;
        g.M = M; g.N = M; g.K = (int)P;
        PCK((gemm<float, float, EPI_STORE>(g, 1, s)), "PCA covariance");
    }
    note_launch();
    pca_random_kernel<<<(unsigned)(((int64_t)M * kp + 255) / 256), 256, 0, s>>>(Q, (int64_t)M * kp, 0x5CA1AB1Eull);
    PCK(cudaGetLastError(), "PCA start");
    std::vector<double> G, Rinv;
    // CholeskyQR2: Qb = orth(Zb) by two steps X <- X R^{-1} with R^T R = X^T X
    // (Zb is overwritten)
    auto orthonormalise = [&](float* Zb, float* Qb) -> tvbx_status {
        if (tvbx_status st = small_product(Zb, Zb, M, kp, dtmp, G, s)) return st;
        if (!chol_inv_upper(G, kp, Rinv))
            return report_error(TVBX_E_NUMERIC, "PCA: basis lost rank (fewer than %d independent FC directions)", kp);
        if (tvbx_status st = right_multiply(Zb, M, kp, Rinv, kp, dS, Qb, s)) return st;
        if (tvbx_status st = small_product(Qb, Qb, M, kp, dtmp, G, s)) return st;
        if (!chol_inv_upper(G, kp, Rinv))
            return report_error(TVBX_E_NUMERIC, "PCA: basis lost rank (fewer than %d independent FC directions)", kp);
        if (tvbx_status st = right_multiply(Qb, M, kp, Rinv, kp, dS, Zb, s)) return st;
        PCK(cudaMemcpyAsync(Qb, Zb, sizeof(float) * M * kp, cudaMemcpyDeviceToDevice, s), "PCA copy");
        return TVBX_OK;
    };
    // orthonormal start, then n_iter steps of Q <- orth(C Q)
    PCK(cudaMemcpyAsync(Z, Q, sizeof(float) * M * kp, cudaMemcpyDeviceToDevice, s), "PCA copy");
    if (tvbx_status st = orthonormalise(Z, Q)) return st;
    for (int it = 0; it < n_iter; ++it) {
        GemmArgs g{};
        g.A = C; g.sam = M; g.sak = 1;
        g.B = Q; g.sbn = 1; g.sbk = kp;
        g.C = Z; g.ldc = kp;
        g.M = M; g.N = kp; g.K = M;
        PCK((gemm<float, float, EPI_STORE>(g, 1, s)), "PCA iteration");
        if (tvbx_status st = orthonormalise(Z, Q)) return st;
    }
    // Rayleigh-Ritz
    {
        GemmArgs g{};
        g.A = C; g.sam = M; g.sak = 1;
        g.B = Q; g.sbn = 1; g.sbk = kp;
        g.C = Z; g.ldc = kp;
        g.M = M; g.N = kp; g.K = M;
        PCK((gemm<float, float, EPI_STORE>(g, 1, s)), "PCA Ritz");
    }
    std::vector<double> H, w, E;
    if (tvbx_status st = small_product(Q, Z, M, kp, dtmp, H, s)) return st;
    for (int i = 0; i < kp; ++i)   // symmetrise
        for (int j = i + 1; j < kp; ++j) {
            const double a = 0.5 * (H[(size_t)i * kp + j] + H[(size_t)j * kp + i]);
            H[(size_t)i * kp + j] = H[(size_t)j * kp + i] = a;
        }
    jacobi_eigen(H, kp, w, E);
    std::vector<int> order(kp);
    std::iota(order.begin(), order.end(), 0);
    std::sort(order.begin(), order.end(), [&](int a, int b) { return w[a] > w[b] || (w[a] == w[b] && a < b); });
    std::vector<double> Esel((size_t)kp * kp, 0.0);   // columns: the n_comp leading eigenvectors
    for (int a = 0; a < kp; ++a)
        for (int c = 0; c < n_comp; ++c) Esel[(size_t)a * kp + c] = E[(size_t)a * kp + order[c]];
    // U^T [n_comp][M]: comps[c][i] = sum_a Q[i][a] E[a][c]
    {
        std::vector<float> h((size_t)kp * kp);
        for (size_t i = 0; i < h.size(); ++i) h[i] = (float)Esel[i];
        PCK(cudaMemcpyAsync(dS, h.data(), sizeof(float) * h.size(), cudaMemcpyHostToDevice, s), "PCA small copy");
        GemmArgs g{};
        g.A = dS; g.sam = 1; g.sak = kp;      // A(m = c, k = a) = E[a][c]
        g.B = Q; g.sbn = kp; g.sbk = 1;       // B(n = i, k = a) = Q[i][a]
        g.C = comps_out; g.ldc = M;
        g.M = n_comp; g.N = M; g.K = kp;
        PCK((gemm<float, float, EPI_STORE>(g, 1, s)), "PCA components");
        PCK(cudaStreamSynchronize(s), "PCA components");
    }
    // sign: largest-magnitude entry positive
    {
        std::vector<float> U((size_t)n_comp * M);
        PCK(cudaMemcpyAsync(U.data(), comps_out, sizeof(float) * U.size(), cudaMemcpyDeviceToHost, s), "PCA sign");
        PCK(cudaStreamSynchronize(s), "PCA sign");
        for (int c = 0; c < n_comp; ++c) {
            float* u = U.data() + (size_t)c * M;
            int am = 0;
            for (int i = 1; i < M; ++i)
                if (fabsf(u[i]) > fabsf(u[am])) am = i;
            if (u[am] < 0.0f)
                for (int i = 0; i < M; ++i) u[i] = -u[i];
        }
        PCK(cudaMemcpyAsync(comps_out, U.data(), sizeof(float) * U.size(), cudaMemcpyHostToDevice, s), "PCA sign");
    }
    if (eigvals_out)
        for (int c = 0; c < n_comp; ++c) eigvals_out[c] = (float)(w[order[c]] / (double)P);
    if (coef_out) {
        GemmArgs g{};
        g.A = V; g.sam = M; g.sak = 1;
        g.B = comps_out; g.sbn = M; g.sbk = 1;
        g.C = coef_out; g.ldc = n_comp;
        g.M = (int)P; g.N = n_comp; g.K = M;
        PCK((gemm<float, float, EPI_STORE>(g, 1, s)), "PCA coefficients");
    }
    PCK(cudaStreamSynchronize(s), "PCA");
    return TVBX_OK;
}

extern "C" tvbx_status tvbx_fc_pca_project(const float* fc, int32_t n_regions, int64_t n_sets, int32_t n_comp,
                                           const float* mean, const float* comps, float* coef_out, void* cuda_stream)
{
    const int N = n_regions;
    const int64_t P = n_sets;
    if (!fc || !mean || !comps || !coef_out) return report_error(TVBX_E_INVALID_ARG, "NULL argument");
    if (N < 3 || N > 512 || P < 1 || P > (1ll << 31) - 1 || n_comp < 1 || n_comp > 64)
        return report_error(TVBX_E_INVALID_ARG, "need 3 <= n_regions <= 512, n_sets >= 1, 1 <= n_comp <= 64");
    const int M = N * (N - 1) / 2;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    DevMem mem(s);
    float* V;
    int2* kj;
    PCK(mem.get(&V, (size_t)P * M), "PCA rows");
    PCK(mem.get(&kj, (size_t)M), "PCA index");
    const std::vector<int2> pairs = triu_pairs(N);
    PCK(cudaMemcpyAsync(kj, pairs.data(), sizeof(int2) * M, cudaMemcpyHostToDevice, s), "PCA index");
    note_launch();
    pca_triu_kernel<<<(unsigned)((P * M + 255) / 256), 256, 0, s>>>(fc, N, P, kj, M, V);
    PCK(cudaGetLastError(), "PCA rows");
    note_launch();
    pca_subtract_kernel<<<(unsigned)((P * M + 255) / 256), 256, 0, s>>>(V, P, M, mean);
    PCK(cudaGetLastError(), "PCA centre");
    GemmArgs g{};
    g.A = V; g.sam = M; g.sak = 1;
    g.B = comps; g.sbn = M; g.sbk = 1;
    g.C = coef_out; g.ldc = n_comp;
    g.M = (int)P; g.N = n_comp; g.K = M;
    PCK((gemm<float, float, EPI_STORE>(g, 1, s)), "PCA coefficients");
    PCK(cudaStreamSynchronize(s), "PCA projection");
    return TVBX_OK;
}

// Host side of the tvbx C-ABI (include/tvbx.h): argument checks, grid
// expansion, delay groups, device memory, chunked launches and exports.

#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "alloc.h"
#include "internal.h"
#include "tvbx.h"

#include <atomic>

using namespace tvbx;

namespace {
std::atomic<uint64_t> g_launches{0};
}

void tvbx::note_launch(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

namespace {

thread_local std::string g_last_error;

tvbx_status fail(tvbx_status code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

}  // namespace

tvbx_status tvbx::report_error(tvbx_status code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

namespace {

tvbx_status cuda_fail(cudaError_t e, const char* what)
{
    if (e == cudaErrorMemoryAllocation)
        return fail(TVBX_E_OOM, "%s: device allocation failed (%s)", what, cudaGetErrorString(e));
    return fail(TVBX_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call, what)                                       \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return cuda_fail(e_, what);   \
    } while (0)

// A device allocation owned by a sweep handle; grows on demand.
// A handle's device buffer, from the allocator in force when it grew
// (tvbx_set_allocator) and released through the same one.
struct DevBuf {
    void* ptr = nullptr;
    size_t bytes = 0;
    DevAllocator how;
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    ~DevBuf() { release(); }
    cudaError_t ensure(size_t n)
    {
        if (n <= bytes && ptr) return cudaSuccess;
        release();
        if (n == 0) return cudaSuccess;
        cudaError_t e = dev_alloc(&ptr, n, &how);
        if (e == cudaSuccess) bytes = n;
        return e;
    }
    void release()
    {
        dev_free(ptr, how);
        ptr = nullptr;
        bytes = 0;
    }
    template <class T> T* as() const { return static_cast<T*>(ptr); }
};

void engine_defaults(tvbx_model* m)
{
    // Table 1 rows as printed (mV), except the RS entry P_sigmaV.tauN, read
    // as -40.7 (with the printed +40.7 the second-order system diverges for
    // every set of the 16-set sweep). Cell, synapse and network constants
    // follow the AdEx mean-field works the paper cites for the model.
    static const double Pe[10] = {-48.9, 5.1, -25.0, 1.4, -0.41, 10.5, -36.0, 7.4, 1.2, -40.7};
    static const double Pi[10] = {-51.4, 0.4, -8.3, 0.2, -0.5, 1.4, -14.6, 4.5, 2.8, 15.3};
    memset(m, 0, sizeof *m);
    const double n_tot = 10000.0, p_conn = 0.05, g_inh = 0.2;
    m->g_L = 10.0; m->C_m = 200.0; m->E_e = 0.0; m->E_i = -80.0;
    m->Q_e = 1.5; m->Q_i = 5.0; m->tau_e = 5.0; m->tau_i = 5.0;
    m->K_e = n_tot * p_conn * (1.0 - g_inh);
    m->K_i = n_tot * p_conn * g_inh;
    m->N_e = n_tot * (1.0 - g_inh);
    m->N_i = n_tot * g_inh;
    m->T = 20.0;
    memcpy(m->P_e, Pe, sizeof Pe);
    memcpy(m->P_i, Pi, sizeof Pi);
    m->mu0 = -60.0; m->dmu0 = 10.0; m->sig0 = 4.0; m->dsig0 = 6.0; m->tau0 = 0.5; m->dtau0 = 1.0;
    m->rate_floor = 1e-9;
    m->tau_OU = 5.0; m->mu_OU = 0.0; m->sigma_OU = 1.0;
    m->b_i = 0.0; m->a_i = 0.0; m->tau_w_i = 1.0;
    m->E_min = 0.0; m->E_max = 0.2;
    m->E0 = 1e-3; m->I0 = 1e-3;
    m->C_div = 1e30;
    double* d = m->defaults;
    d[TVBX_AXIS_G] = 0.0; d[TVBX_AXIS_B_E] = 0.0; d[TVBX_AXIS_TAU_W_E] = 417.0;
    d[TVBX_AXIS_E_L_E] = -64.0; d[TVBX_AXIS_E_L_I] = -64.0; d[TVBX_AXIS_SPEED] = 4.0;
    d[TVBX_AXIS_A_E] = 0.0; d[TVBX_AXIS_W_NOISE] = 1e-6;
    d[TVBX_AXIS_CF_EE] = 0.3e-3; d[TVBX_AXIS_CF_EI] = 0.0; d[TVBX_AXIS_CF_IE] = 0.3e-3;
    d[TVBX_AXIS_CF_II] = 0.0;
}

DevModel to_device_model(const tvbx_model& m, double dt)
{
    DevModel d;
    memset(&d, 0, sizeof d);
    d.g_L = (float)m.g_L; d.C_m = (float)m.C_m; d.E_e = (float)m.E_e; d.E_i = (float)m.E_i;
    d.qe = (float)(m.Q_e * m.tau_e); d.qi = (float)(m.Q_i * m.tau_i);
    d.tau_e = (float)m.tau_e; d.tau_i = (float)m.tau_i;
    d.K_e = (float)m.K_e; d.K_i = (float)m.K_i;
    d.inv_Ne = (float)(1.0 / m.N_e); d.inv_Ni = (float)(1.0 / m.N_i); d.inv_T = (float)(1.0 / m.T);
    for (int i = 0; i < 10; ++i) { d.P_e[i] = (float)m.P_e[i]; d.P_i[i] = (float)m.P_i[i]; }
    d.mu0 = (float)m.mu0; d.inv_dmu0 = (float)(1.0 / m.dmu0);
    d.sig0 = (float)m.sig0; d.inv_dsig0 = (float)(1.0 / m.dsig0);
    d.tau0 = (float)m.tau0; d.inv_dtau0 = (float)(1.0 / m.dtau0);
    d.gL_over_Cm = (float)(m.g_L / m.C_m);
    d.rate_floor = (float)m.rate_floor;
    d.b_i = (float)m.b_i; d.a_i = (float)m.a_i; d.inv_tau_w_i = (float)(1.0 / m.tau_w_i);
    d.E_min = (float)m.E_min; d.E_max = (float)m.E_max;
    d.E0 = (float)m.E0; d.I0 = (float)m.I0;
    d.C_div = (float)std::min(m.C_div, 1e37);
    d.ou_a = (float)(dt / m.tau_OU);
    d.ou_b = (float)(m.sigma_OU * sqrt(dt) / m.tau_OU);
    d.ou_mu = (float)m.mu_OU;
    d.dt = (float)dt;
    // reduced transfer function (tau_e == tau_i): constants of the algebra in
    // model_device.cuh, computed in double and rounded once
    d.reduced = m.tau_e == m.tau_i ? 1 : 0;
    const double qe = m.Q_e * m.tau_e, qi = m.Q_i * m.tau_i, dE = m.E_e - m.E_i;
    const double be = qi * dE, bi = -qe * dE, v1 = 1.0 / m.dmu0, s1 = 1.0 / m.dsig0, z1 = m.g_L / m.dtau0;
    d.tau = (float)m.tau_e;
    d.ke = (float)(qe * qe); d.ki = (float)(qi * qi);
    d.dE = (float)dE;
    d.be = (float)be; d.bi = (float)bi; d.two_be = (float)(2.0 * be); d.two_bi = (float)(2.0 * bi);
    d.gLEe = (float)(m.g_L * m.E_e);
    d.v0 = (float)((m.E_e - m.mu0) * v1); d.v1 = (float)v1;
    d.v1qe = (float)(v1 * qe); d.v1qi = (float)(v1 * qi); d.v1be = (float)(v1 * be); d.two_v1 = (float)(2.0 * v1);
    d.s0 = (float)(m.sig0 * s1); d.s1 = (float)s1; d.s1h = (float)(0.5 * s1); d.s1q = (float)(0.25 * s1);
    d.z0 = (float)((m.tau_e * m.g_L / m.C_m - m.tau0) / m.dtau0); d.z1 = (float)z1;
    d.z1sq = (float)(z1 * z1); d.two_z1 = (float)(2.0 * z1);
    d.sq_e = (float)(2.0 * qe * qe * be * be); d.sq_i = (float)(2.0 * qi * qi * bi * bi);
    // d = theta - mu_V with mu_V = mu0 + dmu0 V, over sqrt(2)
    const double rs2 = 1.0 / sqrt(2.0);
    for (int i = 0; i < 10; ++i) {
        const double ce = m.P_e[i] - (i == 0 ? m.mu0 : 0.0) - (i == 1 ? m.dmu0 : 0.0);
        const double ci = m.P_i[i] - (i == 0 ? m.mu0 : 0.0) - (i == 1 ? m.dmu0 : 0.0);
        d.cp_e[i] = (float)(ce * rs2);
        d.cp_i[i] = (float)(ci * rs2);
    }
    return d;
}

bool model_ok(const tvbx_model& m)
{
    const double pos[] = {m.g_L, m.C_m, m.Q_e, m.Q_i, m.tau_e, m.tau_i, m.K_e, m.K_i, m.N_e, m.N_i,
                          m.T, m.dmu0, m.dsig0, m.dtau0, m.tau_OU, m.tau_w_i};
    for (double v : pos)
        if (!(v > 0.0) || !isfinite(v)) return false;
    return m.E_max > m.E_min && m.C_div > 0.0;
}

int device_ready()
{
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || n < 1) {
        (void)cudaGetLastError();
        return 0;
    }
    return 1;
}

struct Group {
    double speed;
    std::vector<int64_t> sets;      // external indices
    int32_t H = 0;
    std::vector<int32_t> row_ptr;
    std::vector<int32_t> row_mid;   // first zero-delay entry of each row
    std::vector<uint32_t> col_dly;
    std::vector<float> w;
    int64_t ring_offset = 0;        // floats into the ring allocation
    int32_t p_base = 0;
};

}  // namespace

struct tvbx_sweep {
    int32_t N = 0;
    int64_t P = 0;
    std::vector<double> W, L;       // [N][N]
    std::vector<double> prm;        // [P][TVBX_N_AXES], external order
    tvbx_model model;

    // products of the last run
    bool ran = false;
    bool fc_valid = false;
    tvbx_run_cfg cfg{};
    int64_t T = 0;
    cudaStream_t stream = nullptr;
    uint64_t h2d = 0, d2h = 0;      // bytes copied host <-> device
    bool profiling = false;
    std::vector<cudaEvent_t> ev;    // pairs around simulation launches
    size_t ev_used = 0;
    double prof_region_steps = 0.0;
    std::vector<int64_t> perm;      // internal -> external
    std::vector<int64_t> inv;       // external -> internal
    bool identity = true;
    int32_t pb = 16;
    int32_t variant = -1;           // simulation kernel of the last run
    uint64_t gen = 0;               // incremented by every run preparation
    int64_t steps_done = 0;         // steps integrated since the initial state
    bool resumable = false;         // state, ring and OU state hold step steps_done
    int64_t ring_floats = 0;        // size of the ring allocation in use

    DevBuf d_prm, d_ext, d_state, d_status, d_ring, d_series, d_ou_table, d_ou_state;
    DevBuf d_csr_row, d_csr_cd, d_csr_w, d_groups, d_tiles;
    DevBuf d_blocks, d_fc, d_chi, d_meanfc, d_vec, d_fcd, d_tmp, d_perm, d_inv, d_mean_e, d_mean_i, d_error;
    DevBuf d_fcacc, d_shift;        // streamed series: FC moments over the run, fixed shift [N][P]
    DevBuf d_series_i;              // I series (layout sl) when the run keeps it
    SeriesLayout sl{4, 0, 0};      // layout of d_series and d_series_i: set-blocked

    ~tvbx_sweep()
    {
        DevBuf* all[] = {&d_prm, &d_ext, &d_state, &d_status, &d_ring, &d_series, &d_ou_table,
                         &d_ou_state, &d_csr_row, &d_csr_cd, &d_csr_w, &d_groups, &d_tiles,
                         &d_blocks, &d_fc, &d_chi, &d_meanfc, &d_vec, &d_fcd, &d_tmp, &d_perm,
                         &d_inv, &d_mean_e, &d_mean_i, &d_error, &d_fcacc, &d_shift, &d_series_i};
        for (DevBuf* b : all) b->release();
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
    }
};

// ---------------------------------------------------------------------------
// permutation / transposition kernels for exports (internal -> external order)
// ---------------------------------------------------------------------------
__global__ void gather_rows_kernel(const float* __restrict__ in, float* __restrict__ out,
                                   const int64_t* __restrict__ perm, int64_t rows, int64_t len)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < rows * len;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / len, c = i - r * len;
        out[perm[r] * len + c] = in[i];
    }
}
__global__ void gather_u32_kernel(const uint32_t* __restrict__ in, uint32_t* __restrict__ out,
                                  const int64_t* __restrict__ perm, int64_t rows)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < rows;
         i += (int64_t)gridDim.x * blockDim.x)
        out[perm[i]] = in[i];
}
// series in layout sl (internal set order) -> out [np][N][nt] for external sets
// [p0, p0 + np) and samples [t0, t0 + nt); inv maps external -> internal.
__global__ void series_export_kernel(const float* __restrict__ X, const SeriesLayout sl, float* __restrict__ out,
                                     const int64_t* __restrict__ inv, int32_t N, int64_t p0, int64_t np, int64_t t0,
                                     int64_t nt)
{
    const int64_t total = np * N * nt;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = i % nt, rest = i / nt, k = rest % N, q = rest / N;
        out[i] = X[series_index(sl, t0 + t, k, inv[p0 + q])];
    }
}
// state [SV][N][P] -> out [P][8][N]; shared OU from ou_state[k]
__global__ void state_export_kernel(const float* __restrict__ S, const float* __restrict__ ou_state,
                                    float* __restrict__ out, const int64_t* __restrict__ perm, int32_t N,
                                    int64_t P)
{
    const int64_t total = (int64_t)8 * N * P;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = i % P, rest = i / P, k = rest % N, v = rest / N;
        float x = S[i];
        if (v == SV_OU && ou_state) x = ou_state[k];
        out[(perm[p] * 8 + v) * N + k] = x;
    }
}

namespace {

int grid_for(int64_t n) { return (int)std::min<int64_t>((n + 255) / 256, 8192); }

tvbx_status copy_out(void* dst, const void* src, size_t bytes, int32_t mem, cudaStream_t s,
                     uint64_t* d2h_counter = nullptr)
{
    if (bytes == 0) return TVBX_OK;
    if (mem == TVBX_MEM_HOST && d2h_counter) *d2h_counter += bytes;
    CK(cudaMemcpyAsync(dst, src, bytes, mem == TVBX_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s),
       "copy out");
    if (mem == TVBX_MEM_HOST) CK(cudaStreamSynchronize(s), "synchronize");
    return TVBX_OK;
}

// Copy per-set rows (internal order, device) to `dst` in external order.
tvbx_status export_rows(tvbx_sweep* h, const float* src, int64_t len, int32_t mem, float* dst)
{
    const size_t bytes = sizeof(float) * (size_t)h->P * len;
    if (h->identity) return copy_out(dst, src, bytes, mem, h->stream, &h->d2h);
    float* target = dst;
    if (mem == TVBX_MEM_HOST) {
        CK(h->d_tmp.ensure(bytes), "export buffer");
        target = h->d_tmp.as<float>();
    }
    note_launch();
    gather_rows_kernel<<<grid_for(h->P * len), 256, 0, h->stream>>>(src, target, h->d_perm.as<int64_t>(), h->P,
                                                                       len);
    CK(cudaGetLastError(), "gather rows");
    if (mem == TVBX_MEM_HOST) return copy_out(dst, target, bytes, mem, h->stream, &h->d2h);
    return TVBX_OK;
}

// Device errors recorded by the last run's kernels (bounded waits that gave up).
tvbx_status check_device_error(tvbx_sweep* h)
{
    uint32_t err = 0;
    CK(cudaMemcpyAsync(&err, h->d_error.ptr, sizeof err, cudaMemcpyDeviceToHost, h->stream), "error word");
    CK(cudaStreamSynchronize(h->stream), "synchronize");
    if (err & TVBX_DEVERR_TIMEOUT)
        return fail(TVBX_E_TIMEOUT, "a bounded device-side wait (simulation or FC kernel) gave up; results are invalid");
    return TVBX_OK;
}

tvbx_status check_mem(int32_t mem)
{
    if (mem != TVBX_MEM_HOST && mem != TVBX_MEM_DEVICE)
        return fail(TVBX_E_INVALID_ARG, "mem must be TVBX_MEM_HOST or TVBX_MEM_DEVICE");
    return TVBX_OK;
}

tvbx_status create_common(const double* weights, const double* tract_mm, int32_t n_regions,
                          const tvbx_model* model, tvbx_sweep** out, tvbx_sweep** made)
{
    if (!weights || !tract_mm || !out) return fail(TVBX_E_INVALID_ARG, "NULL weights, tract_mm or out");
    if (n_regions < 1 || n_regions > 65535) return fail(TVBX_E_INVALID_ARG, "n_regions must be in [1, 65535]");
    const size_t nn = (size_t)n_regions * n_regions;
    for (size_t i = 0; i < nn; ++i) {
        if (!isfinite(weights[i])) return fail(TVBX_E_INVALID_ARG, "non-finite weight at %zu", i);
        if (!isfinite(tract_mm[i]) || tract_mm[i] < 0.0)
            return fail(TVBX_E_INVALID_ARG, "tract length at %zu must be finite and >= 0", i);
    }
    if (!device_ready()) return fail(TVBX_E_CUDA, "no CUDA device available");
    tvbx_sweep* h = new tvbx_sweep();
    h->N = n_regions;
    h->W.assign(weights, weights + nn);
    h->L.assign(tract_mm, tract_mm + nn);
    if (model) h->model = *model;
    else engine_defaults(&h->model);
    if (!model_ok(h->model)) {
        delete h;
        return fail(TVBX_E_INVALID_ARG, "model constants must be positive where they divide");
    }
    *made = h;
    return TVBX_OK;
}

// Ring row stride: a group's sets rounded up to a multiple of 96 floats, so
// that every tile of 8, 12, 16 or 32 sets lies inside the row and its row
// segment starts on a 16-byte boundary (the alignment TMA bulk copies need).
int64_t ring_stride(size_t sets) { return ((int64_t)sets + 95) / 96 * 96; }

// Build the speed groups for dt: delays, CSR and ring depth per distinct speed.
tvbx_status build_groups(tvbx_sweep* h, double dt, std::vector<Group>& groups)
{
    std::map<double, int> index;
    for (int64_t p = 0; p < h->P; ++p) {
        const double v = h->prm[p * TVBX_N_AXES + TVBX_AXIS_SPEED];
        if (!(v > 0.0) || !isfinite(v)) return fail(TVBX_E_INVALID_ARG, "set %lld: speed must be > 0", (long long)p);
        auto it = index.find(v);
        if (it == index.end()) {
            index[v] = (int)groups.size();
            groups.push_back(Group{});
            groups.back().speed = v;
            it = index.find(v);
        }
        groups[it->second].sets.push_back(p);
    }
    const int N = h->N;
    for (Group& g : groups) {
        g.row_ptr.assign(N + 1, 0);
        g.row_mid.assign(N, 0);
        int64_t dmax = 1;   // ring of at least 3 slots (the padding entries use d = 1)
        for (int k = 0; k < N; ++k) {
            // rows start at an index of the parity of k (zero-weight self entry pads)
            if ((int)(g.col_dly.size() & 1) != (k & 1)) {
                g.col_dly.push_back((1u << 16) | (uint32_t)k);
                g.w.push_back(0.0f);
            }
            g.row_ptr[k] = (int32_t)g.col_dly.size();
            std::vector<std::pair<uint32_t, float>> zero;   // zero-delay entries go last
            for (int j = 0; j < N; ++j) {
                const double w = h->W[(size_t)k * N + j];
                if (w == 0.0) continue;
                // delay in steps: rint (ties to even) of length / (speed dt), in FP64
                const double steps = rint(h->L[(size_t)k * N + j] / (g.speed * dt));
                if (steps > 65533.0) return fail(TVBX_E_UNSUPPORTED, "delay of %g steps exceeds 65533", steps);
                const int64_t d = steps < 0 ? 0 : (int64_t)steps;
                dmax = std::max(dmax, d);
                const uint32_t cd = ((uint32_t)d << 16) | (uint32_t)j;
                if (d == 0) zero.emplace_back(cd, (float)w);
                else { g.col_dly.push_back(cd); g.w.push_back((float)w); }
            }
            g.row_mid[k] = (int32_t)g.col_dly.size();
            for (auto& z : zero) { g.col_dly.push_back(z.first); g.w.push_back(z.second); }
        }
        g.row_ptr[N] = (int32_t)g.col_dly.size();
        g.H = (int32_t)(dmax + 2);
    }
    return TVBX_OK;
}

}  // namespace

extern "C" {

const char* tvbx_version(void) { return "tvbx 0.1 (sm_103a)"; }

const char* tvbx_last_error(void) { return g_last_error.c_str(); }

tvbx_status tvbx_model_defaults(tvbx_model* out)
{
    if (!out) return fail(TVBX_E_INVALID_ARG, "NULL out");
    engine_defaults(out);
    return TVBX_OK;
}

tvbx_status tvbx_sweep_create_points(const double* weights, const double* tract_mm, int32_t n_regions,
                                     int64_t n_sets, const double* params, const tvbx_model* model,
                                     tvbx_sweep** out)
{
    if (n_sets < 1 || n_sets > (int64_t)INT32_MAX) return fail(TVBX_E_INVALID_ARG, "n_sets must be in [1, 2^31)");
    if (!params) return fail(TVBX_E_INVALID_ARG, "NULL params");
    for (int64_t i = 0; i < n_sets * TVBX_N_AXES; ++i)
        if (isinf(params[i])) return fail(TVBX_E_INVALID_ARG, "infinite parameter at %lld", (long long)i);
    tvbx_sweep* h = nullptr;
    tvbx_status st = create_common(weights, tract_mm, n_regions, model, out, &h);
    if (st != TVBX_OK) return st;
    h->P = n_sets;
    h->prm.assign(params, params + n_sets * TVBX_N_AXES);
    *out = h;
    return TVBX_OK;
}

tvbx_status tvbx_sweep_create(const double* weights, const double* tract_mm, int32_t n_regions,
                              const tvbx_grid* grid, const tvbx_model* model, tvbx_sweep** out)
{
    tvbx_model m;
    if (model) m = *model;
    else engine_defaults(&m);
    std::vector<std::vector<double>> vals;
    std::vector<int> axes;
    int64_t P = 1;
    if (grid && grid->n_axes > 0) {
        if (!grid->axes) return fail(TVBX_E_INVALID_ARG, "grid->axes is NULL");
        for (int a = 0; a < grid->n_axes; ++a) {
            const tvbx_axis_spec& s = grid->axes[a];
            if (s.axis < 0 || s.axis >= TVBX_N_AXES) return fail(TVBX_E_INVALID_ARG, "unknown axis %d", s.axis);
            if (std::find(axes.begin(), axes.end(), s.axis) != axes.end())
                return fail(TVBX_E_INVALID_ARG, "axis %d repeated", s.axis);
            if (s.n < 1) return fail(TVBX_E_INVALID_ARG, "axis %d: n must be >= 1", s.axis);
            std::vector<double> v((size_t)s.n);
            for (int i = 0; i < s.n; ++i) {
                if (s.values) v[i] = s.values[i];
                else v[i] = s.n > 1 ? s.lo + (s.hi - s.lo) * (double)i / (double)(s.n - 1) : s.lo;
            }
            axes.push_back(s.axis);
            vals.push_back(v);
            P *= s.n;
            if (P > (int64_t)INT32_MAX) return fail(TVBX_E_INVALID_ARG, "grid has more than 2^31 sets");
        }
    }
    std::vector<double> prm((size_t)P * TVBX_N_AXES);
    for (int64_t p = 0; p < P; ++p) {
        double* row = prm.data() + p * TVBX_N_AXES;
        for (int a = 0; a < TVBX_N_AXES; ++a) row[a] = m.defaults[a];
        int64_t rem = p;
        for (int a = (int)axes.size() - 1; a >= 0; --a) {   // last axis fastest
            const int64_t n = (int64_t)vals[a].size();
            row[axes[a]] = vals[a][rem % n];
            rem /= n;
        }
    }
    return tvbx_sweep_create_points(weights, tract_mm, n_regions, P, prm.data(), &m, out);
}

tvbx_status tvbx_sweep_info(const tvbx_sweep* h, int64_t* n_sets, int32_t* n_regions, int64_t* n_samples)
{
    if (!h) return fail(TVBX_E_INVALID_ARG, "NULL handle");
    if (n_sets) *n_sets = h->P;
    if (n_regions) *n_regions = h->N;
    if (n_samples) *n_samples = h->ran ? h->T : 0;
    return TVBX_OK;
}

// Everything a run needs before its first simulation launch: argument
// checks, delay groups, internal set order, kernel and tile choice, device
// buffers and uploads; with device_init also the state and ring
// initialisation on stream s. general_pb > 0 forces the general kernel (or,
// with direct_body, the register-tile body) with that tile width (batches).
struct RunPlan {
    SimArgs a;
    int variant = -1;
    int pb = 16;
    int32_t n_tiles = 0;
    int nnz_max = 0;
    int64_t chunk = 0;
    std::vector<GroupDev> gdev;
    std::vector<TileDev> tiles;
    std::vector<int64_t> tile_nnz;   // weights per row of the tile's group (cost model)
};

// n_base > 0: the run continues a trajectory at global step n_base (state,
// ring buffers and OU state are kept; the series and the running sums start
// afresh for the new samples).
static tvbx_status prepare_run(tvbx_sweep* h, const tvbx_run_cfg& c, cudaStream_t s, int general_pb,
                               bool device_init, RunPlan& plan, bool direct_body = false, int64_t n_base = 0)
{
    if (!(c.dt_ms > 0.0) || !isfinite(c.dt_ms)) return fail(TVBX_E_INVALID_ARG, "dt_ms must be > 0");
    if (c.n_steps < 0 || n_base + c.n_steps > ((int64_t)1 << 32) - 2)
        return fail(TVBX_E_INVALID_ARG, "steps so far plus n_steps must be in [0, 2^32 - 1)");
    if (c.tavg_steps < 1) return fail(TVBX_E_INVALID_ARG, "tavg_steps must be >= 1");
    if (c.chunk_steps < 0 || (c.chunk_steps > 0 && c.chunk_steps % c.tavg_steps != 0))
        return fail(TVBX_E_INVALID_ARG, "chunk_steps must be 0 or a positive multiple of tavg_steps");
    const int64_t T = c.n_steps / c.tavg_steps;
    if (c.transient_samples < 0 || (T > 0 && c.transient_samples >= T))
        return fail(TVBX_E_INVALID_ARG, "transient_samples must be in [0, n_samples)");
    if (c.p_offset < 0) return fail(TVBX_E_INVALID_ARG, "p_offset must be >= 0");
    if (c.series_mode != TVBX_SERIES_KEEP && c.series_mode != TVBX_SERIES_STREAM)
        return fail(TVBX_E_INVALID_ARG, "unknown series_mode %d", c.series_mode);
    if (c.series_mode == TVBX_SERIES_STREAM && h->N > 384)
        return fail(TVBX_E_UNSUPPORTED, "a streamed series needs n_regions <= 384 (have %d)", h->N);
    if (c.keep_i_series != 0 && c.keep_i_series != 1)
        return fail(TVBX_E_INVALID_ARG, "keep_i_series must be 0 or 1");
    if (c.keep_i_series && c.series_mode != TVBX_SERIES_KEEP)
        return fail(TVBX_E_INVALID_ARG, "keep_i_series needs series_mode TVBX_SERIES_KEEP");
    h->stream = s;
    h->ran = false;
    h->fc_valid = false;
    h->resumable = false;
    h->gen += 1;

    std::vector<Group> groups;
    tvbx_status st = build_groups(h, c.dt_ms, groups);
    if (st != TVBX_OK) return st;
    const int N = h->N;
    const int64_t P = h->P;

    // internal order: sets grouped by speed
    h->perm.clear();
    int64_t ring_floats = 0;
    for (Group& g : groups) {
        g.p_base = (int32_t)h->perm.size();
        ring_floats = (ring_floats + 63) / 64 * 64;   // 256-byte aligned ring per group
        g.ring_offset = ring_floats;
        ring_floats += (int64_t)g.H * N * ring_stride(g.sets.size());
        for (int64_t e : g.sets) h->perm.push_back(e);
    }
    h->identity = true;
    for (int64_t i = 0; i < P; ++i)
        if (h->perm[i] != i) { h->identity = false; break; }

    // per-set parameters in internal order, SoA
    std::vector<float> prm_soa((size_t)TVBX_N_AXES * P);
    for (int64_t i = 0; i < P; ++i)
        for (int a = 0; a < TVBX_N_AXES; ++a)
            prm_soa[(size_t)a * P + i] = (float)h->prm[h->perm[i] * TVBX_N_AXES + a];

    // kernel and tile size: the prefetching kernel when its shared-memory
    // gather buffer fits, else the general kernel
    int nnz_max = 0;
    for (const Group& g : groups) nnz_max = std::max(nnz_max, (int)g.col_dly.size());
    if (c.kernel != TVBX_KERNEL_DIRECT &&
        (c.kernel < TVBX_KERNEL_AUTO || c.kernel >= TVBX_KERNEL_PREFETCH + sim_fast_variants()))
        return fail(TVBX_E_INVALID_ARG, "unknown kernel %d", c.kernel);
    if (c.withhold_step < 0) return fail(TVBX_E_INVALID_ARG, "withhold_step must be >= 0");
    int variant = -1;   // prefetch variant, -1 = general kernel, -2 = register-tile kernel
    if (general_pb > 0) {
        // batch: the batch's body and tile width
        if (direct_body) variant = -2;
    } else if (c.kernel == TVBX_KERNEL_AUTO) {
        // preference order from measurement on the 32,768-set, 68-region sweep
        // (the packed kernels, slower there, need the reduced transfer
        // function, tau_e == tau_i); connectomes too large for the prefetch
        // buffer take the register tiles
        const bool reduced = h->model.tau_e == h->model.tau_i;
        for (int v : {15, 0, 1, 2, 3, 9, 8})
            if ((reduced || !sim_fast_packed(v)) && sim_fast_fits(v, N, nnz_max)) { variant = v; break; }
        if (variant < 0 && sim_direct_pb(N) > 0) variant = -2;
    } else if (c.kernel == TVBX_KERNEL_DIRECT) {
        if (sim_direct_pb(N) == 0) return fail(TVBX_E_UNSUPPORTED, "register-tile kernel: too many regions (%d)", N);
        variant = -2;
    } else if (c.kernel != TVBX_KERNEL_GENERAL) {
        variant = c.kernel - TVBX_KERNEL_PREFETCH;
        if (sim_fast_packed(variant) && h->model.tau_e != h->model.tau_i)
            return fail(TVBX_E_UNSUPPORTED, "packed kernel %d needs tau_e == tau_i", c.kernel);
        if (!sim_fast_fits(variant, N, nnz_max))
            return fail(TVBX_E_UNSUPPORTED, "prefetch kernel %d does not fit %d regions / %d weights", c.kernel, N,
                        nnz_max);
    }
    int pb = 16;
    if (general_pb > 0) {
        pb = general_pb;
        if (!direct_body && sim_smem_bytes(N, pb) > 227 * 1024)
            return fail(TVBX_E_UNSUPPORTED, "n_regions %d too large", N);
    } else if (variant >= 0) {
        pb = sim_fast_pb(variant);
    } else if (variant == -2) {
        pb = sim_direct_pb(N);
    } else {
        while (pb > 8 && sim_smem_bytes(N, pb) > 200 * 1024) pb /= 2;
        if (sim_smem_bytes(N, pb) > 200 * 1024) return fail(TVBX_E_UNSUPPORTED, "n_regions %d too large", N);
    }
    h->pb = pb;
    h->variant = variant;
    std::vector<TileDev> tiles;
    std::vector<GroupDev> gdev(groups.size());
    std::vector<int32_t> all_row;
    std::vector<uint32_t> all_cd;
    std::vector<float> all_w;
    std::vector<int64_t> row_off(groups.size()), nz_off(groups.size());
    for (size_t gi = 0; gi < groups.size(); ++gi) {
        Group& g = groups[gi];
        row_off[gi] = (int64_t)all_row.size();
        nz_off[gi] = (int64_t)all_cd.size();
        all_row.insert(all_row.end(), g.row_ptr.begin(), g.row_ptr.end());
        all_row.insert(all_row.end(), g.row_mid.begin(), g.row_mid.end());
        all_cd.insert(all_cd.end(), g.col_dly.begin(), g.col_dly.end());
        all_w.insert(all_w.end(), g.w.begin(), g.w.end());
        const int32_t Pg = (int32_t)g.sets.size();
        for (int32_t q0 = 0; q0 < Pg; q0 += pb) {
            tiles.push_back(TileDev{(int32_t)gi, q0, std::min(pb, Pg - q0), 0});
            plan.tile_nnz.push_back((int64_t)g.col_dly.size());
        }
    }
    if (all_cd.empty()) { all_cd.push_back(0); all_w.push_back(0.f); }

    // chunking: keep each launch around 4-8 thousand steps
    int64_t chunk = c.chunk_steps > 0 ? c.chunk_steps : 0;
    if (chunk == 0) {
        chunk = (int64_t)c.tavg_steps * std::max<int64_t>(1, 5000 / c.tavg_steps);
        if (chunk <= 0) chunk = c.tavg_steps;
    }
    chunk = std::min<int64_t>(chunk, std::max<int64_t>(c.n_steps, 1));
    // a streamed series keeps the samples of one chunk (rounded up to whole samples)
    const int64_t series_T =
        c.series_mode == TVBX_SERIES_STREAM ? std::min<int64_t>(T, (chunk + c.tavg_steps - 1) / c.tavg_steps) : T;

    // device memory
    CK(h->d_prm.ensure(sizeof(float) * prm_soa.size()), "parameters");
    CK(h->d_ext.ensure(sizeof(int64_t) * P), "set index");
    CK(h->d_perm.ensure(sizeof(int64_t) * P), "set index");
    CK(h->d_inv.ensure(sizeof(int64_t) * P), "set index");
    CK(h->d_state.ensure(sizeof(float) * (size_t)SV_COUNT * N * P), "state");
    CK(h->d_status.ensure(sizeof(uint32_t) * P), "status");
    CK(h->d_ring.ensure(sizeof(float) * (size_t)std::max<int64_t>(ring_floats, 1)), "ring buffers");
    // set-blocked series: groups of 4 sets, [ceil(P / 4)][series_T][N][4]
    const int64_t P4 = (P + 3) / 4 * 4;
    h->sl = layout_blocked(N, std::max<int64_t>(series_T, 1));
    CK(h->d_series.ensure(sizeof(float) * (size_t)std::max<int64_t>(series_T * N * P4, 1)), "series");
    if (c.keep_i_series)
        CK(h->d_series_i.ensure(sizeof(float) * (size_t)std::max<int64_t>(T * N * P4, 1)), "I series");
    if (c.series_mode == TVBX_SERIES_STREAM) {
        CK(h->d_fcacc.ensure(sizeof(float) * (size_t)P * ((size_t)N * N + N)), "streamed FC moments");
        CK(h->d_blocks.ensure(sizeof(float) * (size_t)P * ((size_t)N * N + N)), "FC block moments");
        CK(h->d_shift.ensure(sizeof(float) * (size_t)N * P), "FC shift");
    }
    CK(h->d_ou_state.ensure(sizeof(float) * N), "OU state");
    CK(h->d_error.ensure(sizeof(uint32_t)), "error word");
    CK(h->d_csr_row.ensure(sizeof(int32_t) * all_row.size()), "CSR");
    CK(h->d_csr_cd.ensure(sizeof(uint32_t) * all_cd.size()), "CSR");
    CK(h->d_csr_w.ensure(sizeof(float) * all_w.size()), "CSR");
    CK(h->d_groups.ensure(sizeof(GroupDev) * gdev.size()), "groups");
    CK(h->d_tiles.ensure(sizeof(TileDev) * std::max<size_t>(tiles.size(), 1)), "tiles");
    for (size_t gi = 0; gi < groups.size(); ++gi) {
        GroupDev& d = gdev[gi];
        d.ring = h->d_ring.as<float>() + groups[gi].ring_offset;
        d.row_ptr = h->d_csr_row.as<int32_t>() + row_off[gi];
        d.row_mid = h->d_csr_row.as<int32_t>() + row_off[gi] + N + 1;
        d.col_dly = h->d_csr_cd.as<uint32_t>() + nz_off[gi];
        d.w = h->d_csr_w.as<float>() + nz_off[gi];
        d.H = groups[gi].H;
        d.P_g = (int32_t)groups[gi].sets.size();
        d.p_base = groups[gi].p_base;
        d.stride = (int32_t)ring_stride(groups[gi].sets.size());
        d.nnz = (int32_t)groups[gi].col_dly.size();
        d.nnz_d = 0;
        for (uint32_t cd : groups[gi].col_dly) d.nnz_d += (cd >> 16) != 0;
    }
    h->h2d += sizeof(float) * prm_soa.size() + 3 * sizeof(int64_t) * P + sizeof(int32_t) * all_row.size() +
              sizeof(uint32_t) * all_cd.size() + sizeof(float) * all_w.size() + sizeof(GroupDev) * gdev.size() +
              sizeof(TileDev) * tiles.size();
    CK(cudaMemcpyAsync(h->d_prm.ptr, prm_soa.data(), sizeof(float) * prm_soa.size(), cudaMemcpyHostToDevice, s), "upload");
    CK(cudaMemcpyAsync(h->d_ext.ptr, h->perm.data(), sizeof(int64_t) * P, cudaMemcpyHostToDevice, s), "upload");
    CK(cudaMemcpyAsync(h->d_perm.ptr, h->perm.data(), sizeof(int64_t) * P, cudaMemcpyHostToDevice, s), "upload");
    h->inv.assign((size_t)P, 0);
    for (int64_t i = 0; i < P; ++i) h->inv[h->perm[i]] = i;
    CK(cudaMemcpyAsync(h->d_inv.ptr, h->inv.data(), sizeof(int64_t) * P, cudaMemcpyHostToDevice, s), "upload");
    CK(cudaMemcpyAsync(h->d_csr_row.ptr, all_row.data(), sizeof(int32_t) * all_row.size(), cudaMemcpyHostToDevice, s), "upload");
    CK(cudaMemcpyAsync(h->d_csr_cd.ptr, all_cd.data(), sizeof(uint32_t) * all_cd.size(), cudaMemcpyHostToDevice, s), "upload");
    CK(cudaMemcpyAsync(h->d_csr_w.ptr, all_w.data(), sizeof(float) * all_w.size(), cudaMemcpyHostToDevice, s), "upload");
    CK(cudaMemcpyAsync(h->d_groups.ptr, gdev.data(), sizeof(GroupDev) * gdev.size(), cudaMemcpyHostToDevice, s), "upload");
    if (!tiles.empty())
        CK(cudaMemcpyAsync(h->d_tiles.ptr, tiles.data(), sizeof(TileDev) * tiles.size(), cudaMemcpyHostToDevice, s), "upload");
    if (n_base == 0) CK(cudaMemsetAsync(h->d_ou_state.ptr, 0, sizeof(float) * N, s), "OU state");
    CK(cudaMemsetAsync(h->d_error.ptr, 0, sizeof(uint32_t), s), "error word");
    h->ring_floats = ring_floats;

    if (!c.noise_per_set) CK(h->d_ou_table.ensure(sizeof(float) * (size_t)chunk * N), "OU table");

    SimArgs a;
    memset(&a, 0, sizeof a);
    a.m = to_device_model(h->model, c.dt_ms);
    a.groups = h->d_groups.as<GroupDev>();
    a.tiles = h->d_tiles.as<TileDev>();
    a.prm = h->d_prm.as<float>();
    a.ext_index = h->d_ext.as<int64_t>();
    a.state = h->d_state.as<float>();
    a.series = h->d_series.as<float>();
    a.sl = h->sl;
    a.series_i = c.keep_i_series ? h->d_series_i.as<float>() : nullptr;
    a.ou_table = c.noise_per_set ? nullptr : h->d_ou_table.as<float>();
    a.status = h->d_status.as<uint32_t>();
    a.error = h->d_error.as<uint32_t>();
    a.withhold_step = c.withhold_step > 0 ? (int64_t)c.withhold_step - 1 : -1;
    a.wait_limit = c.withhold_step > 0 ? (1u << 12) : (1u << 26);
    a.N = N;
    a.P = (int32_t)P;
    a.ts = c.tavg_steps;
    a.T = T;
    a.transient = c.transient_samples;
    a.noise_per_set = c.noise_per_set ? 1 : 0;
    a.seed = c.seed;
    a.p_offset = c.p_offset;
    if (n_base > 0) {
        // the kernels index samples by the global step, t = (n + 1) / ts - 1:
        // shift the window [t_base, t_base + T) onto the series buffer (the
        // address is formed in integers; every write lands inside the buffer)
        const int64_t t_base = n_base / c.tavg_steps;
        a.series = reinterpret_cast<float*>(reinterpret_cast<uintptr_t>(h->d_series.ptr) -
                                            (uintptr_t)(sizeof(float) * (size_t)t_base * h->sl.st));
        if (c.keep_i_series)
            a.series_i = reinterpret_cast<float*>(reinterpret_cast<uintptr_t>(h->d_series_i.ptr) -
                                                  (uintptr_t)(sizeof(float) * (size_t)t_base * h->sl.st));
        a.T = t_base + T;
        a.transient = t_base + c.transient_samples;
        // running sums (means, FC shift) cover the new samples only
        CK(cudaMemsetAsync(h->d_state.as<float>() + (size_t)SV_SUM_E * N * P, 0,
                           sizeof(float) * (size_t)(SV_CMP_I - SV_SUM_E + 1) * N * P, s),
           "running sums");
    }

    if (device_init) {
        CK(launch_init_state(a, s), "init state");
        for (size_t gi = 0; gi < groups.size(); ++gi)
            CK(launch_init_ring(gdev[gi].ring, (int64_t)gdev[gi].H * N * gdev[gi].stride, a.m.E0, s), "init ring");
    }
    plan.a = a;
    plan.variant = variant;
    plan.pb = pb;
    plan.n_tiles = (int32_t)tiles.size();
    plan.nnz_max = nnz_max;
    plan.chunk = chunk;
    plan.gdev = gdev;
    plan.tiles = tiles;
    return TVBX_OK;
}

// Mark a handle's run as complete (results may be read). steps_before: the
// global step the run started at; resumable: the state may be continued.
static void finish_run(tvbx_sweep* h, const tvbx_run_cfg& c, int64_t steps_before = 0, bool resumable = false)
{
    h->cfg = c;
    h->T = c.n_steps / c.tavg_steps;
    h->ran = true;
    h->fc_valid = false;   // a relaunched batch graph rewrites the status words, and the FC pass adds to them
    h->steps_done = steps_before + c.n_steps;
    h->resumable = resumable;
}

// Streamed series: fold the samples after the transient of the chunk of
// steps [n0, n0 + n_chunk), held in the series buffer from its row 0, into
// the run's FC moments. The shift of every chunk is the one taken from the
// first chunk with such samples (shift_set), so that the moments add.
static tvbx_status stream_fc_chunk(tvbx_sweep* h, const SimArgs& a, int64_t n0, int32_t n_chunk, bool& shift_set,
                                   cudaStream_t s)
{
    const int64_t tc0 = n0 / a.ts, tc1 = (n0 + n_chunk) / a.ts;   // global samples of the chunk
    const int64_t u0 = std::max<int64_t>(tc0, a.transient);
    if (u0 >= tc1) return TVBX_OK;
    const float* buf = h->d_series.as<float>();
    if (!shift_set) {
        CK(launch_fc_shift(buf, h->sl, a.N, a.P, u0 - tc0, tc1 - tc0, h->d_shift.as<float>(), s), "FC shift");
        shift_set = true;
    }
    FcArgs f;
    memset(&f, 0, sizeof f);
    f.series = buf;
    f.sl = h->sl;
    f.shift = h->d_shift.as<float>();
    f.N = a.N;
    f.P = a.P;
    f.t_begin = u0 - tc0;
    f.t_end = tc1 - tc0;
    f.n_blocks = 1;
    f.blocks = h->d_blocks.as<float>();
    f.status = h->d_status.as<uint32_t>();
    f.error = h->d_error.as<uint32_t>();
    f.wait_limit = 1u << 22;
    CK(launch_fc_moments(f, s), "streamed FC moments");
    CK(launch_fc_accumulate(f.blocks, h->d_fcacc.as<float>(), (int64_t)a.P * ((int64_t)a.N * a.N + a.N), s),
       "streamed FC moments");
    return TVBX_OK;
}

// The series pointer of a chunk whose first sample t0 goes to row 0 of the
// buffer (the kernels index samples by the global step; the address is
// formed in integers and every write lands inside the buffer).
static float* series_at(void* buf, int64_t t0, const SeriesLayout& sl)
{
    return reinterpret_cast<float*>(reinterpret_cast<uintptr_t>(buf) - (uintptr_t)(sizeof(float) * (size_t)t0 * sl.st));
}

// Enqueue the chunked launches of a prepared run over global steps
// [n_base, n_base + c.n_steps).
static tvbx_status run_chunks(tvbx_sweep* h, const tvbx_run_cfg& c, const RunPlan& plan, int64_t n_base,
                              cudaStream_t s)
{
    SimArgs a = plan.a;
    const int N = h->N;
    const int64_t P = h->P;
    const int64_t chunk = plan.chunk;
    const int variant = plan.variant;
    const bool streamed = c.series_mode == TVBX_SERIES_STREAM;
    bool shift_set = false;
    if (streamed)
        CK(cudaMemsetAsync(h->d_fcacc.ptr, 0, sizeof(float) * (size_t)P * ((size_t)N * N + N), s),
           "streamed FC moments");
    for (int64_t n0 = n_base; n0 < n_base + c.n_steps; n0 += chunk) {
        a.n0 = n0;
        a.n_chunk = (int32_t)std::min<int64_t>(chunk, n_base + c.n_steps - n0);
        if (streamed) a.series = series_at(h->d_series.ptr, n0 / c.tavg_steps, h->sl);
        if (!c.noise_per_set)
            CK(launch_ou_table(a.m, h->d_ou_table.as<float>(), h->d_ou_state.as<float>(), N, n0, a.n_chunk, c.seed, s),
               "OU table");
        if (h->profiling) {
            while (h->ev.size() < h->ev_used + 2) {
                cudaEvent_t e;
                CK(cudaEventCreate(&e), "profiling event");
                h->ev.push_back(e);
            }
            CK(cudaEventRecord(h->ev[h->ev_used], s), "profiling event");
        }
        if (variant >= 0) CK(launch_sim_fast(a, variant, plan.n_tiles, plan.nnz_max, s), "simulation chunk");
        else if (variant == -2) CK(launch_sim_direct(a, plan.n_tiles, plan.pb, s), "simulation chunk");
        else CK(launch_sim_chunk(a, plan.n_tiles, plan.pb, s), "simulation chunk");
        if (h->profiling) {
            CK(cudaEventRecord(h->ev[h->ev_used + 1], s), "profiling event");
            h->ev_used += 2;
            h->prof_region_steps += (double)P * N * a.n_chunk;
        }
        if (streamed)
            if (tvbx_status st = stream_fc_chunk(h, a, n0, a.n_chunk, shift_set, s)) return st;
    }
    return TVBX_OK;
}

tvbx_status tvbx_run(tvbx_sweep* h, const tvbx_run_cfg* cfg, void* cuda_stream)
{
    if (!h || !cfg) return fail(TVBX_E_INVALID_ARG, "NULL handle or cfg");
    const tvbx_run_cfg c = *cfg;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    RunPlan plan;
    tvbx_status st = prepare_run(h, c, s, 0, true, plan);
    if (st != TVBX_OK) return st;
    if ((st = run_chunks(h, c, plan, 0, s)) != TVBX_OK) return st;
    finish_run(h, c, 0, true);
    return TVBX_OK;
}

tvbx_status tvbx_run_continue(tvbx_sweep* h, int64_t n_steps, int32_t transient_samples, void* cuda_stream)
{
    if (!h) return fail(TVBX_E_INVALID_ARG, "NULL handle");
    if (!h->resumable) return fail(TVBX_E_BAD_STATE, "tvbx_run_continue needs a completed tvbx_run, "
                                                     "tvbx_run_continue or tvbx_restore on this handle");
    tvbx_run_cfg c = h->cfg;
    if (h->steps_done % c.tavg_steps != 0)
        return fail(TVBX_E_BAD_STATE, "the steps so far (%lld) are not a multiple of tavg_steps (%d)",
                    (long long)h->steps_done, c.tavg_steps);
    if (n_steps < 0) return fail(TVBX_E_INVALID_ARG, "n_steps must be >= 0");
    c.n_steps = n_steps;
    c.transient_samples = transient_samples;
    const int64_t n_base = h->steps_done;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    RunPlan plan;
    tvbx_status st = prepare_run(h, c, s, 0, false, plan, false, n_base);
    if (st != TVBX_OK) return st;
    if ((st = run_chunks(h, c, plan, n_base, s)) != TVBX_OK) return st;
    finish_run(h, c, n_base, true);
    return TVBX_OK;
}

// ---------------------------------------------------------------------------
// checkpoint / restore
// ---------------------------------------------------------------------------
namespace {

constexpr char CKPT_MAGIC[8] = {'T', 'V', 'B', 'X', 'C', 'K', 'P', '3'};   // 3: W carries, series mode

struct CkptHeader {
    char magic[8];
    uint64_t fingerprint;     // of the sweep's connectome, points and constants
    int64_t n_regions;
    int64_t n_sets;
    int64_t steps_done;
    int64_t ring_floats;
    double dt_ms;
    int64_t tavg_steps;
    int64_t noise_per_set;
    uint64_t seed;
    int64_t p_offset;
    int64_t chunk_steps;
    int64_t kernel;
    int64_t series_mode;
    int64_t keep_i_series;
};

// FNV-1a over the bytes of the definition of a sweep (all fields are doubles
// or integers without padding)
uint64_t sweep_fingerprint(const tvbx_sweep* h)
{
    uint64_t x = 1469598103934665603ull;
    auto mix = [&](const void* p, size_t n) {
        const unsigned char* b = static_cast<const unsigned char*>(p);
        for (size_t i = 0; i < n; ++i) x = (x ^ b[i]) * 1099511628211ull;
    };
    const int64_t dims[2] = {h->N, h->P};
    mix(dims, sizeof dims);
    mix(h->W.data(), sizeof(double) * h->W.size());
    mix(h->L.data(), sizeof(double) * h->L.size());
    mix(h->prm.data(), sizeof(double) * h->prm.size());
    mix(&h->model, sizeof h->model);
    return x;
}

size_t ckpt_bytes(int64_t N, int64_t P, int64_t ring_floats)
{
    return sizeof(CkptHeader) + sizeof(float) * ((size_t)SV_COUNT * N * P + (size_t)ring_floats + (size_t)N) +
           sizeof(uint32_t) * (size_t)P;
}

}  // namespace

tvbx_status tvbx_checkpoint_size(const tvbx_sweep* h, uint64_t* bytes)
{
    if (!h || !bytes) return fail(TVBX_E_INVALID_ARG, "NULL handle or bytes");
    if (!h->resumable) return fail(TVBX_E_BAD_STATE, "nothing to checkpoint: no completed run on this handle");
    *bytes = ckpt_bytes(h->N, h->P, h->ring_floats);
    return TVBX_OK;
}

tvbx_status tvbx_checkpoint(tvbx_sweep* h, void* host_buf, uint64_t bytes)
{
    if (!h || !host_buf) return fail(TVBX_E_INVALID_ARG, "NULL handle or buffer");
    if (!h->resumable) return fail(TVBX_E_BAD_STATE, "nothing to checkpoint: no completed run on this handle");
    const int64_t N = h->N, P = h->P;
    const size_t need = ckpt_bytes(N, P, h->ring_floats);
    if (bytes < need) return fail(TVBX_E_INVALID_ARG, "checkpoint buffer holds %llu bytes, needs %zu",
                                  (unsigned long long)bytes, need);
    CK(cudaStreamSynchronize(h->stream), "checkpoint");
    if (tvbx_status e = check_device_error(h)) return e;
    CkptHeader hd;
    memset(&hd, 0, sizeof hd);
    memcpy(hd.magic, CKPT_MAGIC, sizeof hd.magic);
    hd.fingerprint = sweep_fingerprint(h);
    hd.n_regions = N;
    hd.n_sets = P;
    hd.steps_done = h->steps_done;
    hd.ring_floats = h->ring_floats;
    hd.dt_ms = h->cfg.dt_ms;
    hd.tavg_steps = h->cfg.tavg_steps;
    hd.noise_per_set = h->cfg.noise_per_set;
    hd.seed = h->cfg.seed;
    hd.p_offset = h->cfg.p_offset;
    hd.chunk_steps = h->cfg.chunk_steps;
    hd.kernel = h->cfg.kernel;
    hd.series_mode = h->cfg.series_mode;
    hd.keep_i_series = h->cfg.keep_i_series;
    unsigned char* out = static_cast<unsigned char*>(host_buf);
    memcpy(out, &hd, sizeof hd);
    size_t off = sizeof hd;
    const size_t b_state = sizeof(float) * (size_t)SV_COUNT * N * P;
    const size_t b_status = sizeof(uint32_t) * (size_t)P;
    const size_t b_ring = sizeof(float) * (size_t)h->ring_floats;
    const size_t b_ou = sizeof(float) * (size_t)N;
    CK(cudaMemcpy(out + off, h->d_state.ptr, b_state, cudaMemcpyDeviceToHost), "checkpoint state");
    off += b_state;
    CK(cudaMemcpy(out + off, h->d_status.ptr, b_status, cudaMemcpyDeviceToHost), "checkpoint status");
    off += b_status;
    if (b_ring) CK(cudaMemcpy(out + off, h->d_ring.ptr, b_ring, cudaMemcpyDeviceToHost), "checkpoint ring");
    off += b_ring;
    CK(cudaMemcpy(out + off, h->d_ou_state.ptr, b_ou, cudaMemcpyDeviceToHost), "checkpoint OU state");
    h->d2h += need - sizeof hd;
    return TVBX_OK;
}

tvbx_status tvbx_restore(tvbx_sweep* h, const void* host_buf, uint64_t bytes)
{
    if (!h || !host_buf) return fail(TVBX_E_INVALID_ARG, "NULL handle or buffer");
    if (bytes < sizeof(CkptHeader)) return fail(TVBX_E_INVALID_ARG, "checkpoint too short");
    CkptHeader hd;
    memcpy(&hd, host_buf, sizeof hd);
    if (memcmp(hd.magic, CKPT_MAGIC, sizeof hd.magic) != 0) return fail(TVBX_E_INVALID_ARG, "not a tvbx checkpoint");
    if (hd.n_regions != h->N || hd.n_sets != h->P || hd.fingerprint != sweep_fingerprint(h))
        return fail(TVBX_E_INVALID_ARG, "checkpoint of a different sweep (connectome, points or constants differ)");
    if (hd.ring_floats < 0 || hd.steps_done < 0 || bytes < ckpt_bytes(h->N, h->P, hd.ring_floats))
        return fail(TVBX_E_INVALID_ARG, "checkpoint truncated");
    tvbx_run_cfg c;
    memset(&c, 0, sizeof c);
    c.dt_ms = hd.dt_ms;
    c.n_steps = 0;
    c.tavg_steps = (int32_t)hd.tavg_steps;
    c.noise_per_set = (int32_t)hd.noise_per_set;
    c.seed = hd.seed;
    c.p_offset = hd.p_offset;
    c.chunk_steps = (int32_t)hd.chunk_steps;
    c.kernel = (int32_t)hd.kernel;
    c.series_mode = (int32_t)hd.series_mode;
    c.keep_i_series = (int32_t)hd.keep_i_series;
    // lay out the buffers as the checkpointed run did, then fill them; the
    // handle's earlier stream may no longer exist, so the device is drained
    // and the default stream used
    CK(cudaDeviceSynchronize(), "restore");
    RunPlan plan;
    tvbx_status st = prepare_run(h, c, nullptr, 0, false, plan);
    if (st != TVBX_OK) return st;
    if (h->ring_floats != hd.ring_floats) return fail(TVBX_E_INVALID_ARG, "checkpoint ring layout differs");
    const int64_t N = h->N, P = h->P;
    const unsigned char* in = static_cast<const unsigned char*>(host_buf) + sizeof hd;
    const size_t b_state = sizeof(float) * (size_t)SV_COUNT * N * P;
    const size_t b_status = sizeof(uint32_t) * (size_t)P;
    const size_t b_ring = sizeof(float) * (size_t)hd.ring_floats;
    const size_t b_ou = sizeof(float) * (size_t)N;
    CK(cudaStreamSynchronize(nullptr), "restore");
    CK(cudaMemcpy(h->d_state.ptr, in, b_state, cudaMemcpyHostToDevice), "restore state");
    in += b_state;
    CK(cudaMemcpy(h->d_status.ptr, in, b_status, cudaMemcpyHostToDevice), "restore status");
    in += b_status;
    if (b_ring) CK(cudaMemcpy(h->d_ring.ptr, in, b_ring, cudaMemcpyHostToDevice), "restore ring");
    in += b_ring;
    CK(cudaMemcpy(h->d_ou_state.ptr, in, b_ou, cudaMemcpyHostToDevice), "restore OU state");
    h->h2d += b_state + b_status + b_ring + b_ou;
    h->cfg = c;
    h->T = 0;
    h->ran = false;
    h->steps_done = hd.steps_done;
    h->resumable = true;
    return TVBX_OK;
}

static tvbx_status run_fc(tvbx_sweep* h, int32_t precision, int32_t fcd_window, int32_t fcd_step, int32_t* nw_out)
{
    const int N = h->N;
    const int64_t P = h->P;
    const int64_t t0 = h->cfg.transient_samples, t1 = h->T;
    const int64_t Tn = t1 - t0;
    if (Tn < 1) return fail(TVBX_E_BAD_STATE, "the last run produced no samples");
    int32_t blk = 0, n_blocks = 1, m = 0, nw = 0;
    if (fcd_window > 0) {
        if (fcd_step < 1 || fcd_window % fcd_step != 0)
            return fail(TVBX_E_INVALID_ARG, "fcd_window must be a positive multiple of fcd_step");
        if (fcd_window > Tn) return fail(TVBX_E_INVALID_ARG, "fcd_window exceeds the samples after the transient");
        if (N < 3) return fail(TVBX_E_INVALID_ARG, "FCD needs at least 3 regions");
        blk = fcd_step;
        n_blocks = (int32_t)((Tn + blk - 1) / blk);
        m = fcd_window / fcd_step;
        nw = (int32_t)((Tn - fcd_window) / fcd_step + 1);
    }
    const size_t stride_b = (size_t)N * N + N;
    if (h->cfg.series_mode == TVBX_SERIES_STREAM) {
        // the moments were folded chunk by chunk during the run
        if (fcd_window > 0)
            return fail(TVBX_E_INVALID_ARG, "the FCD needs the whole series, and the last run streamed it");
        CK(h->d_fc.ensure(sizeof(float) * (size_t)P * N * N), "FC");
        CK(h->d_chi.ensure(sizeof(float) * P), "chi");
        CK(h->d_meanfc.ensure(sizeof(float) * P), "mean FC");
        FcArgs f;
        memset(&f, 0, sizeof f);
        f.N = N;
        f.P = (int32_t)P;
        f.t_begin = t0;
        f.t_end = t1;
        f.n_blocks = 1;
        f.blocks = h->d_fcacc.as<float>();
        f.fc = h->d_fc.as<float>();
        f.chi = h->d_chi.as<float>();
        f.mean_fc = h->d_meanfc.as<float>();
        f.status = h->d_status.as<uint32_t>();
        f.error = h->d_error.as<uint32_t>();
        f.wait_limit = 1u << 22;
        CK(launch_fc_reduce(f, 0, 0, 0, nullptr, nullptr, h->stream), "FC reduction");
        if (nw_out) *nw_out = 0;
        h->fc_valid = true;
        return TVBX_OK;
    }
    CK(h->d_blocks.ensure(sizeof(float) * (size_t)P * n_blocks * stride_b), "FC block moments");
    CK(h->d_fc.ensure(sizeof(float) * (size_t)P * N * N), "FC");
    CK(h->d_chi.ensure(sizeof(float) * P), "chi");
    CK(h->d_meanfc.ensure(sizeof(float) * P), "mean FC");
    FcArgs f;
    memset(&f, 0, sizeof f);
    f.series = h->d_series.as<float>();
    f.sl = h->sl;
    f.state = h->d_state.as<float>();
    f.N = N;
    f.P = (int32_t)P;
    f.t_begin = t0;
    f.t_end = t1;
    f.blk = blk;
    f.n_blocks = n_blocks;
    f.blocks = h->d_blocks.as<float>();
    f.fc = h->d_fc.as<float>();
    f.chi = h->d_chi.as<float>();
    f.mean_fc = h->d_meanfc.as<float>();
    f.status = h->d_status.as<uint32_t>();
    f.error = h->d_error.as<uint32_t>();
    f.wait_limit = 1u << 22;
    if (precision == TVBX_FC_FP32) CK(launch_fc_moments(f, h->stream), "FC moments");
    else CK(launch_fc_tc_moments(f, precision, h->stream), "FC tensor-core moments");
    float* vec = nullptr;
    float* fcd = nullptr;
    if (fcd_window > 0) {
        const size_t M = (size_t)N * (N - 1) / 2;
        if (fc_reduce_needs_vec_scratch(N, n_blocks, nw)) {
            CK(h->d_vec.ensure(sizeof(float) * (size_t)P * nw * M), "FCD vectors");
            vec = h->d_vec.as<float>();
        }
        CK(h->d_fcd.ensure(sizeof(float) * (size_t)P * nw * nw), "FCD");
        fcd = h->d_fcd.as<float>();
    }
    CK(launch_fc_reduce(f, m, nw, fcd_window, vec, fcd, h->stream), "FC / FCD reduction");
    if (nw_out) *nw_out = nw;
    h->fc_valid = true;
    return TVBX_OK;
}

tvbx_status tvbx_fc(tvbx_sweep* h, const tvbx_fc_cfg* cfg, int32_t mem, float* fc_out, float* fcd_out,
                    int32_t* n_windows)
{
    if (!h || !cfg) return fail(TVBX_E_INVALID_ARG, "NULL handle or cfg");
    if (check_mem(mem)) return TVBX_E_INVALID_ARG;
    if (!h->ran) return fail(TVBX_E_BAD_STATE, "tvbx_fc before tvbx_run");
    if (tvbx_status e = check_device_error(h)) return e;
    if (cfg->precision < TVBX_FC_FP32 || cfg->precision > TVBX_FC_TF32X3)
        return fail(TVBX_E_UNSUPPORTED, "FC precision %d", cfg->precision);
    if (cfg->precision != TVBX_FC_FP32 && h->cfg.series_mode != TVBX_SERIES_STREAM &&
        !fc_tc_supported(h->N, cfg->precision))
        return fail(TVBX_E_INVALID_ARG, "tensor-core FC needs n_regions <= 112 (have %d)", h->N);
    if (cfg->fcd_window < 0) return fail(TVBX_E_INVALID_ARG, "fcd_window must be >= 0");
    int32_t nw = 0;
    tvbx_status st = run_fc(h, cfg->precision, cfg->fcd_window, cfg->fcd_step, &nw);
    if (st != TVBX_OK) return st;
    if (cfg->precision != TVBX_FC_FP32 && h->cfg.series_mode != TVBX_SERIES_STREAM &&
        (st = check_device_error(h)) != TVBX_OK)
        return st;
    if (n_windows) *n_windows = nw;
    if (fc_out) {
        st = export_rows(h, h->d_fc.as<float>(), (int64_t)h->N * h->N, mem, fc_out);
        if (st != TVBX_OK) return st;
    }
    if (fcd_out && cfg->fcd_window > 0) {
        st = export_rows(h, h->d_fcd.as<float>(), (int64_t)nw * nw, mem, fcd_out);
        if (st != TVBX_OK) return st;
    }
    if (mem == TVBX_MEM_HOST) CK(cudaStreamSynchronize(h->stream), "synchronize");
    return TVBX_OK;
}

namespace {
// Stream-ordered pool of the FC scratch of tvbx_fc_series, one per device,
// owned by the library: it keeps freed memory for the next call instead of
// returning it to the driver (so repeated calls do not re-map gigabytes).
std::mutex g_pool_mu;
cudaMemPool_t g_pools[64] = {};

cudaError_t scratch_pool(cudaMemPool_t* out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_pool_mu);
    if (!g_pools[dev]) {
        cudaMemPoolProps props;
        memset(&props, 0, sizeof props);
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool;
        if ((e = cudaMemPoolCreate(&pool, &props)) != cudaSuccess) return e;
        uint64_t keep = UINT64_MAX;
        if ((e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep)) != cudaSuccess) return e;
        g_pools[dev] = pool;
    }
    *out = g_pools[dev];
    return cudaSuccess;
}
}  // namespace

tvbx_status tvbx_fc_series(const float* series, int32_t n_regions, int64_t n_sets, int64_t n_samples,
                           const tvbx_fc_cfg* cfg, float* fc_out, float* fcd_out, int32_t* n_windows, float* chi,
                           float* mean_fc, uint32_t* set_status, void* cuda_stream)
{
    if (!series || !cfg) return fail(TVBX_E_INVALID_ARG, "NULL series or cfg");
    const int N = n_regions;
    const int64_t P = n_sets, Tn = n_samples;
    if (N < 1 || P < 1 || Tn < 1) return fail(TVBX_E_INVALID_ARG, "sizes must be >= 1");
    if (P > (int64_t)INT32_MAX) return fail(TVBX_E_INVALID_ARG, "n_sets must be < 2^31");
    if (cfg->precision < TVBX_FC_FP32 || cfg->precision > TVBX_FC_TF32X3)
        return fail(TVBX_E_UNSUPPORTED, "FC precision %d", cfg->precision);
    if (cfg->precision != TVBX_FC_FP32 && !fc_tc_supported(N, cfg->precision))
        return fail(TVBX_E_INVALID_ARG, "tensor-core FC needs n_regions <= 112 (have %d)", N);
    if (cfg->precision == TVBX_FC_FP32 && N > 384) return fail(TVBX_E_INVALID_ARG, "FC needs n_regions <= 384");
    int32_t blk = 0, n_blocks = 1, m = 0, nw = 0;
    if (cfg->series_layout != TVBX_LAYOUT_TNP && cfg->series_layout != TVBX_LAYOUT_SET4)
        return fail(TVBX_E_INVALID_ARG, "unknown series_layout %d", cfg->series_layout);
    const SeriesLayout sl = cfg->series_layout == TVBX_LAYOUT_SET4 ? layout_blocked(N, Tn) : layout_tnp(N, P);
    if (cfg->fcd_window < 0) return fail(TVBX_E_INVALID_ARG, "fcd_window must be >= 0");
    if (cfg->fcd_window > 0) {
        if (cfg->fcd_step < 1 || cfg->fcd_window % cfg->fcd_step != 0)
            return fail(TVBX_E_INVALID_ARG, "fcd_window must be a positive multiple of fcd_step");
        if (cfg->fcd_window > Tn) return fail(TVBX_E_INVALID_ARG, "fcd_window exceeds n_samples");
        if (N < 3) return fail(TVBX_E_INVALID_ARG, "FCD needs at least 3 regions");
        blk = cfg->fcd_step;
        n_blocks = (int32_t)((Tn + blk - 1) / blk);
        m = cfg->fcd_window / cfg->fcd_step;
        nw = (int32_t)((Tn - cfg->fcd_window) / cfg->fcd_step + 1);
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const size_t stride_b = (size_t)N * N + N;
    const size_t M = (size_t)N * (N - 1) / 2;
    const size_t sz_blocks = sizeof(float) * (size_t)P * n_blocks * stride_b;
    const size_t sz_shift = sizeof(float) * (size_t)N * P;
    const size_t sz_fc = fc_out ? 0 : sizeof(float) * (size_t)P * N * N;
    const size_t sz_small = sizeof(float) * (size_t)P * 3 + 256;
    const size_t sz_vec = nw > 0 && fc_reduce_needs_vec_scratch(N, n_blocks, nw) ? sizeof(float) * (size_t)P * nw * M : 0;
    const size_t sz_fcd = (nw > 0 && !fcd_out) ? sizeof(float) * (size_t)P * nw * nw : 0;
    auto up = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t total = up(sz_blocks) + up(sz_shift) + up(sz_fc) + up(sz_small) + up(sz_vec) + up(sz_fcd);
    void* scratch = nullptr;
    cudaMemPool_t pool;
    CK(scratch_pool(&pool), "FC scratch pool");
    CK(cudaMallocFromPoolAsync(&scratch, total, pool, s), "FC scratch");
    char* q = static_cast<char*>(scratch);
    auto take = [&](size_t b) { char* r = q; q += up(b); return r; };
    float* d_blocks = reinterpret_cast<float*>(take(sz_blocks));
    float* d_shift = reinterpret_cast<float*>(take(sz_shift));
    float* d_fc = fc_out ? fc_out : reinterpret_cast<float*>(take(sz_fc));
    char* small = take(sz_small);
    float* d_chi = chi ? chi : reinterpret_cast<float*>(small);
    float* d_mfc = mean_fc ? mean_fc : reinterpret_cast<float*>(small) + P;
    uint32_t* d_status = set_status ? set_status : reinterpret_cast<uint32_t*>(reinterpret_cast<float*>(small) + 2 * P);
    uint32_t* d_err = reinterpret_cast<uint32_t*>(reinterpret_cast<float*>(small) + 3 * P);
    float* d_vec = sz_vec > 0 ? reinterpret_cast<float*>(take(sz_vec)) : nullptr;
    float* d_fcd = nw > 0 ? (fcd_out ? fcd_out : reinterpret_cast<float*>(take(sz_fcd))) : nullptr;

    tvbx_status st = TVBX_OK;
    cudaError_t e = cudaSuccess;
    do {
        if ((e = cudaMemsetAsync(small, 0, sz_small, s)) != cudaSuccess) break;
        if ((e = launch_fc_shift(series, sl, N, P, 0, Tn, d_shift, s)) != cudaSuccess) break;
        FcArgs f;
        memset(&f, 0, sizeof f);
        f.series = series;
        f.sl = sl;
        f.state = nullptr;
        f.shift = d_shift;
        f.N = N;
        f.P = (int32_t)P;
        f.t_begin = 0;
        f.t_end = Tn;
        f.blk = blk;
        f.n_blocks = n_blocks;
        f.blocks = d_blocks;
        f.fc = d_fc;
        f.chi = d_chi;
        f.mean_fc = d_mfc;
        f.status = d_status;
        f.error = d_err;
        f.wait_limit = 1u << 22;
        if (cfg->precision == TVBX_FC_FP32) e = launch_fc_moments(f, s);
        else e = launch_fc_tc_moments(f, cfg->precision, s);
        if (e != cudaSuccess) break;
        if ((e = launch_fc_reduce(f, m, nw, cfg->fcd_window, d_vec, d_fcd, s)) != cudaSuccess) break;
    } while (0);
    uint32_t err = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&err, d_err, sizeof err, cudaMemcpyDeviceToHost, s);
    cudaError_t ef = cudaFreeAsync(scratch, s);
    cudaError_t es = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_fail(e, "FC of series");
    else if (ef != cudaSuccess) st = cuda_fail(ef, "FC scratch free");
    else if (es != cudaSuccess) st = cuda_fail(es, "synchronize");
    else if (err & TVBX_DEVERR_TIMEOUT)
        st = fail(TVBX_E_TIMEOUT, "a bounded device-side wait of the FC kernel gave up; results are invalid");
    if (st == TVBX_OK && n_windows) *n_windows = nw;
    return st;
}

tvbx_status tvbx_summary(tvbx_sweep* h, int32_t mem, float* mean_e_hz, float* mean_i_hz, float* chi,
                         float* mean_fc, uint32_t* status)
{
    if (!h) return fail(TVBX_E_INVALID_ARG, "NULL handle");
    if (check_mem(mem)) return TVBX_E_INVALID_ARG;
    if (!h->ran) return fail(TVBX_E_BAD_STATE, "tvbx_summary before tvbx_run");
    if (tvbx_status e = check_device_error(h)) return e;
    const int64_t P = h->P;
    if ((chi || mean_fc || status) && !h->fc_valid) {
        tvbx_status st = run_fc(h, TVBX_FC_FP32, 0, 0, nullptr);
        if (st != TVBX_OK) return st;
    }
    tvbx_status st = TVBX_OK;
    if (mean_e_hz || mean_i_hz) {
        CK(h->d_mean_e.ensure(sizeof(float) * P), "summary");
        CK(h->d_mean_i.ensure(sizeof(float) * P), "summary");
        CK(launch_summary(h->d_state.as<float>(), h->N, (int32_t)P, h->T - h->cfg.transient_samples,
                          h->d_mean_e.as<float>(), h->d_mean_i.as<float>(), h->stream),
           "summary");
        if (mean_e_hz && (st = export_rows(h, h->d_mean_e.as<float>(), 1, mem, mean_e_hz))) return st;
        if (mean_i_hz && (st = export_rows(h, h->d_mean_i.as<float>(), 1, mem, mean_i_hz))) return st;
    }
    if (chi && (st = export_rows(h, h->d_chi.as<float>(), 1, mem, chi))) return st;
    if (mean_fc && (st = export_rows(h, h->d_meanfc.as<float>(), 1, mem, mean_fc))) return st;
    if (status) {
        uint32_t* target = status;
        if (!h->identity) {
            CK(h->d_tmp.ensure(sizeof(uint32_t) * P), "export buffer");
            target = mem == TVBX_MEM_HOST ? h->d_tmp.as<uint32_t>() : status;
            note_launch();
            gather_u32_kernel<<<grid_for(P), 256, 0, h->stream>>>(h->d_status.as<uint32_t>(), target,
                                                                   h->d_perm.as<int64_t>(), P);
            CK(cudaGetLastError(), "gather status");
            if (mem == TVBX_MEM_HOST && (st = copy_out(status, target, sizeof(uint32_t) * P, mem, h->stream, &h->d2h))) return st;
        } else if ((st = copy_out(status, h->d_status.ptr, sizeof(uint32_t) * P, mem, h->stream, &h->d2h))) {
            return st;
        }
    }
    if (mem == TVBX_MEM_HOST) CK(cudaStreamSynchronize(h->stream), "synchronize");
    return TVBX_OK;
}

tvbx_status tvbx_series_pop_range(const tvbx_sweep* hc, int32_t pop, int64_t set_begin, int64_t set_count,
                                  int64_t t_begin, int64_t t_count, int32_t mem, float* out)
{
    tvbx_sweep* h = const_cast<tvbx_sweep*>(hc);
    if (!h || !out) return fail(TVBX_E_INVALID_ARG, "NULL handle or out");
    if (pop != 0 && pop != 1) return fail(TVBX_E_INVALID_ARG, "pop must be 0 (E) or 1 (I)");
    if (check_mem(mem)) return TVBX_E_INVALID_ARG;
    if (!h->ran) return fail(TVBX_E_BAD_STATE, "series export before tvbx_run");
    if (h->cfg.series_mode == TVBX_SERIES_STREAM)
        return fail(TVBX_E_BAD_STATE, "the last run streamed its series (series_mode): there is none to export");
    if (pop == 1 && !h->cfg.keep_i_series)
        return fail(TVBX_E_BAD_STATE, "the last run kept no I series (keep_i_series)");
    if (tvbx_status e = check_device_error(h)) return e;
    if (set_begin < 0 || set_count < 0 || set_begin + set_count > h->P || t_begin < 0 || t_count < 0 ||
        t_begin + t_count > h->T)
        return fail(TVBX_E_INVALID_ARG, "series window outside [0, %lld) x [0, %lld)", (long long)h->P,
                    (long long)h->T);
    const size_t total = (size_t)set_count * h->N * t_count;
    if (total == 0) return TVBX_OK;
    float* target = out;
    if (mem == TVBX_MEM_HOST) {
        CK(h->d_tmp.ensure(sizeof(float) * total), "export buffer");
        target = h->d_tmp.as<float>();
    }
    note_launch();
    series_export_kernel<<<grid_for((int64_t)total), 256, 0, h->stream>>>(
        (pop ? h->d_series_i : h->d_series).as<float>(), h->sl, target, h->d_inv.as<int64_t>(), h->N, set_begin,
        set_count, t_begin, t_count);
    CK(cudaGetLastError(), "series export");
    if (mem == TVBX_MEM_HOST) return copy_out(out, target, sizeof(float) * total, mem, h->stream, &h->d2h);
    return TVBX_OK;
}

tvbx_status tvbx_series_range(const tvbx_sweep* h, int64_t set_begin, int64_t set_count, int64_t t_begin,
                              int64_t t_count, int32_t mem, float* out)
{
    return tvbx_series_pop_range(h, 0, set_begin, set_count, t_begin, t_count, mem, out);
}

tvbx_status tvbx_series(const tvbx_sweep* h, int32_t mem, float* out)
{
    if (!h) return fail(TVBX_E_INVALID_ARG, "NULL handle");
    return tvbx_series_range(h, 0, h->P, 0, h->T, mem, out);
}

tvbx_status tvbx_state(const tvbx_sweep* hc, int32_t mem, float* out)
{
    tvbx_sweep* h = const_cast<tvbx_sweep*>(hc);
    if (!h || !out) return fail(TVBX_E_INVALID_ARG, "NULL handle or out");
    if (check_mem(mem)) return TVBX_E_INVALID_ARG;
    if (!h->ran) return fail(TVBX_E_BAD_STATE, "tvbx_state before tvbx_run");
    if (tvbx_status e = check_device_error(h)) return e;
    const size_t total = (size_t)8 * h->N * h->P;
    float* target = out;
    if (mem == TVBX_MEM_HOST) {
        CK(h->d_tmp.ensure(sizeof(float) * total), "export buffer");
        target = h->d_tmp.as<float>();
    }
    note_launch();
    state_export_kernel<<<grid_for((int64_t)total), 256, 0, h->stream>>>(
        h->d_state.as<float>(), h->cfg.noise_per_set ? nullptr : h->d_ou_state.as<float>(), target,
        h->d_perm.as<int64_t>(), h->N, h->P);
    CK(cudaGetLastError(), "state export");
    if (mem == TVBX_MEM_HOST) return copy_out(out, target, sizeof(float) * total, mem, h->stream, &h->d2h);
    return TVBX_OK;
}

tvbx_status tvbx_transfer_function(const tvbx_model* model, int32_t pop, int64_t n, int32_t mem,
                                   const float* x_e, const float* x_i, const float* W, const float* E_L,
                                   const float* C, float* out)
{
    if (pop != 0 && pop != 1) return fail(TVBX_E_INVALID_ARG, "pop must be 0 or 1");
    if (n < 0) return fail(TVBX_E_INVALID_ARG, "n must be >= 0");
    if (check_mem(mem)) return TVBX_E_INVALID_ARG;
    if (n == 0) return TVBX_OK;
    if (!x_e || !x_i || !W || !E_L || !out) return fail(TVBX_E_INVALID_ARG, "NULL array");
    if (!device_ready()) return fail(TVBX_E_CUDA, "no CUDA device available");
    tvbx_model m;
    if (model) m = *model;
    else engine_defaults(&m);
    if (!model_ok(m)) return fail(TVBX_E_INVALID_ARG, "model constants must be positive where they divide");
    const DevModel dm = to_device_model(m, 0.1);
    DevBuf in, res;
    const float *dxe = x_e, *dxi = x_i, *dW = W, *dEL = E_L, *dC = C;
    float* dout = out;
    if (mem == TVBX_MEM_HOST) {
        CK(in.ensure(sizeof(float) * 7 * n), "inputs");
        CK(res.ensure(sizeof(float) * 8 * n), "outputs");
        float* b = in.as<float>();
        CK(cudaMemcpy(b, x_e, sizeof(float) * n, cudaMemcpyHostToDevice), "upload");
        CK(cudaMemcpy(b + n, x_i, sizeof(float) * n, cudaMemcpyHostToDevice), "upload");
        CK(cudaMemcpy(b + 2 * n, W, sizeof(float) * n, cudaMemcpyHostToDevice), "upload");
        CK(cudaMemcpy(b + 3 * n, E_L, sizeof(float) * n, cudaMemcpyHostToDevice), "upload");
        if (C) CK(cudaMemcpy(b + 4 * n, C, sizeof(float) * 3 * n, cudaMemcpyHostToDevice), "upload");
        dxe = b; dxi = b + n; dW = b + 2 * n; dEL = b + 3 * n; dC = C ? b + 4 * n : nullptr;
        dout = res.as<float>();
    }
    CK(launch_tf_eval(dm, pop, n, dxe, dxi, dW, dEL, dC, dout, 0), "transfer function");
    if (mem == TVBX_MEM_HOST) CK(cudaMemcpy(out, dout, sizeof(float) * 8 * n, cudaMemcpyDeviceToHost), "download");
    CK(cudaDeviceSynchronize(), "synchronize");
    in.release();
    res.release();
    return TVBX_OK;
}

uint64_t tvbx_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

tvbx_status tvbx_last_kernel(const tvbx_sweep* h, int32_t* kernel, int32_t* sets_per_tile)
{
    if (!h) return fail(TVBX_E_INVALID_ARG, "NULL handle");
    if (!h->ran) return fail(TVBX_E_BAD_STATE, "tvbx_last_kernel before tvbx_run");
    if (kernel)
        *kernel = h->variant == -2 ? TVBX_KERNEL_DIRECT
                                   : (h->variant < 0 ? TVBX_KERNEL_GENERAL : TVBX_KERNEL_PREFETCH + h->variant);
    if (sets_per_tile) *sets_per_tile = h->pb;
    return TVBX_OK;
}

tvbx_status tvbx_transfer_bytes(const tvbx_sweep* h, uint64_t* h2d, uint64_t* d2h)
{
    if (!h) return fail(TVBX_E_INVALID_ARG, "NULL handle");
    if (h2d) *h2d = h->h2d;
    if (d2h) *d2h = h->d2h;
    return TVBX_OK;
}

tvbx_status tvbx_profile_enable(tvbx_sweep* h, int32_t enable)
{
    if (!h) return fail(TVBX_E_INVALID_ARG, "NULL handle");
    if (h->stream) CK(cudaStreamSynchronize(h->stream), "synchronize");
    h->profiling = enable != 0;
    h->ev_used = 0;
    h->prof_region_steps = 0.0;
    return TVBX_OK;
}

tvbx_status tvbx_profile_read(tvbx_sweep* h, double* sim_ms, int64_t* sim_launches, double* region_steps)
{
    if (!h) return fail(TVBX_E_INVALID_ARG, "NULL handle");
    CK(cudaStreamSynchronize(h->stream), "synchronize");
    double total = 0.0;
    for (size_t i = 0; i + 1 < h->ev_used; i += 2) {
        float ms = 0.0f;
        CK(cudaEventElapsedTime(&ms, h->ev[i], h->ev[i + 1]), "event time");
        total += ms;
    }
    if (sim_ms) *sim_ms = total;
    if (sim_launches) *sim_launches = (int64_t)(h->ev_used / 2);
    if (region_steps) *region_steps = h->prof_region_steps;
    return TVBX_OK;
}

tvbx_status tvbx_sweep_destroy(tvbx_sweep* h)
{
    if (!h) return TVBX_OK;
    if (h->stream) cudaStreamSynchronize(h->stream);
    delete h;
    return TVBX_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batches of sweeps: one persistent launch, captured in a CUDA graph
// ---------------------------------------------------------------------------
struct tvbx_batch {
    std::vector<tvbx_sweep*> jobs;
    std::vector<tvbx_run_cfg> cfgs;
    std::vector<uint64_t> gens;     // generation of each job when the graph was built
    std::vector<tvbx_run_cfg> cfgs_run;   // configurations the graph runs (trial runs are shorter)
    cudaStream_t stream = nullptr;
    int32_t threads = 512;
    size_t smem_budget = 200 * 1024;
    bool direct = false;                // register-tile bodies where a job fits
    bool only_direct = false;           // every job on register tiles
    DevBuf d_jobs, d_items, d_head, d_ou;
    int32_t n_items = 0, grid = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t graph_nodes = 0, graph_kernels = 0;
    bool built = false;

    void drop_graph()
    {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        exec = nullptr;
        graph = nullptr;
        built = false;
    }
    ~tvbx_batch()
    {
        drop_graph();
        d_jobs.release();
        d_items.release();
        d_head.release();
        d_ou.release();
        if (stream) cudaStreamDestroy(stream);
    }
};

namespace {

// Tile width of a job under a shared-memory budget: the widest of 32, 16, 8
// sets whose state fits.
int batch_pb(int N, size_t budget, int threads)
{
    for (int pb : {32, 16, 8})
        if (sim_smem_bytes(N, pb) <= budget && threads % pb == 0) return pb;
    return 0;
}

// Prepare every job (tile width from the budget; trial_steps > 0 shortens
// each job), build the LPT-ordered work list, and capture the device work of
// one run -- per-job state, ring and OU-table initialisation, the queue reset
// and the persistent kernel -- in a CUDA graph.
// Work enqueued on a job's own stream must finish before the batch's stream
// (non-blocking: it does not order with the legacy default stream) touches
// the job's buffers.
tvbx_status batch_adopt_jobs(tvbx_batch* b)
{
    for (tvbx_sweep* h : b->jobs)
        if (h->stream != b->stream) {
            CK(cudaStreamSynchronize(h->stream), "job stream");
            h->stream = b->stream;
        }
    return TVBX_OK;
}

tvbx_status batch_build(tvbx_batch* b, int32_t threads, size_t budget, int64_t trial_steps, bool direct)
{
    b->drop_graph();
    if (tvbx_status st = batch_adopt_jobs(b)) return st;
    const size_t nj = b->jobs.size();
    std::vector<RunPlan> plans(nj);
    std::vector<tvbx_run_cfg> run_cfgs(b->cfgs);
    std::vector<int> pbs(nj), dirs(nj);
    size_t smem = 0;
    int64_t ou_floats = 0;
    std::vector<int64_t> ou_off(nj, -1);
    // streamed series: the batch runs in rounds of S steps, the streamed jobs'
    // common chunk, and folds each round's samples into their FC moments
    int64_t S = 0;
    for (size_t j = 0; j < nj; ++j) {
        const tvbx_run_cfg& c = b->cfgs[j];
        if (c.series_mode != TVBX_SERIES_STREAM) continue;
        const int64_t cj =
            c.chunk_steps > 0 ? c.chunk_steps : (int64_t)c.tavg_steps * std::max<int64_t>(1, 5000 / c.tavg_steps);
        if (S == 0) S = cj;
        if (cj != S)
            return fail(TVBX_E_INVALID_ARG, "batch job %zu: streamed jobs share one chunk (%lld steps, have %lld)", j,
                        (long long)S, (long long)cj);
    }
    for (size_t j = 0; j < nj && S > 0; ++j)
        if (S % b->cfgs[j].tavg_steps != 0)
            return fail(TVBX_E_INVALID_ARG, "batch job %zu: tavg_steps must divide the streamed chunk of %lld steps", j,
                        (long long)S);
    for (size_t j = 0; j < nj; ++j) {
        tvbx_run_cfg& c = run_cfgs[j];
        if (trial_steps > 0) {   // timing run only: shortened, no transient
            c.n_steps = std::min<int64_t>(c.n_steps, std::max<int64_t>(trial_steps / c.tavg_steps, 1) * c.tavg_steps);
            c.transient_samples = 0;
        }
        if (c.n_steps > INT32_MAX) return fail(TVBX_E_INVALID_ARG, "batch job %zu: n_steps must be < 2^31", j);
        const int N = b->jobs[j]->N;
        // register tiles: as many 4-set quads per region as the CTA has threads for
        const bool dj = direct && N <= threads;
        const int pb = dj ? 4 * (threads / N) : batch_pb(N, budget, threads);
        if (!pb) return fail(TVBX_E_UNSUPPORTED, "batch job %zu: %d regions do not fit %zu bytes of shared memory", j,
                             N, budget);
        pbs[j] = pb;
        dirs[j] = dj ? 1 : 0;
        smem = std::max(smem, dj ? sizeof(float) * 11 * (size_t)pb : sim_smem_bytes(N, pb));
        c.chunk_steps = c.series_mode == TVBX_SERIES_STREAM ? (int32_t)S : 0;
        tvbx_status st = prepare_run(b->jobs[j], c, b->stream, pb, false, plans[j], dj);
        if (st != TVBX_OK) return st;
        if (!c.noise_per_set) {
            ou_off[j] = ou_floats;
            ou_floats += ((int64_t)c.n_steps * b->jobs[j]->N + 63) / 64 * 64;
        }
    }
    CK(b->d_ou.ensure(sizeof(float) * (size_t)std::max<int64_t>(ou_floats, 1)), "batch OU tables");
    int64_t max_steps = 0;
    for (size_t j = 0; j < nj; ++j) max_steps = std::max<int64_t>(max_steps, run_cfgs[j].n_steps);
    const int64_t R = S > 0 ? (max_steps + S - 1) / S : 1;   // rounds
    const int64_t round_steps = S > 0 ? S : max_steps;
    std::vector<BatchJob> jobs((size_t)R * nj);               // [round][job]
    struct Cost { double c; int32_t job, tile; };
    std::vector<BatchItem> items;
    std::vector<int64_t> item_off((size_t)R + 1, 0);
    for (int64_t r = 0; r < R; ++r) {
        std::vector<Cost> costs;
        for (size_t j = 0; j < nj; ++j) {
            const int64_t n0 = r * round_steps, nc = std::min<int64_t>(round_steps, run_cfgs[j].n_steps - n0);
            SimArgs a = plans[j].a;
            a.n0 = n0;
            a.n_chunk = (int32_t)std::max<int64_t>(nc, 0);
            a.ou_table = ou_off[j] >= 0 ? b->d_ou.as<float>() + ou_off[j] + n0 * b->jobs[j]->N : nullptr;
            if (run_cfgs[j].series_mode == TVBX_SERIES_STREAM)
                a.series = series_at(b->jobs[j]->d_series.ptr, n0 / run_cfgs[j].tavg_steps, b->jobs[j]->sl);
            jobs[(size_t)r * nj + j] = BatchJob{a, pbs[j], dirs[j]};
            if (nc <= 0) continue;
            const int N = b->jobs[j]->N;
            for (int32_t t = 0; t < plans[j].n_tiles; ++t) {
                const double per_step = (double)N * 40.0 + (double)plans[j].tile_nnz[t];   // TF work + gathers
                costs.push_back(Cost{per_step * (double)nc * plans[j].tiles[t].nq, (int32_t)(r * nj + j), t});
            }
        }
        std::stable_sort(costs.begin(), costs.end(), [](const Cost& x, const Cost& y) { return x.c > y.c; });
        for (const Cost& c : costs) items.push_back(BatchItem{c.job, c.tile});
        item_off[(size_t)r + 1] = (int64_t)items.size();
    }
    b->n_items = (int32_t)items.size();
    CK(b->d_jobs.ensure(sizeof(BatchJob) * jobs.size()), "batch jobs");
    CK(b->d_items.ensure(sizeof(BatchItem) * std::max<size_t>(items.size(), 1)), "batch items");
    CK(b->d_head.ensure(sizeof(int32_t) * (size_t)R), "batch queue");
    CK(cudaMemcpyAsync(b->d_jobs.ptr, jobs.data(), sizeof(BatchJob) * jobs.size(), cudaMemcpyHostToDevice, b->stream),
       "upload");
    if (!items.empty())
        CK(cudaMemcpyAsync(b->d_items.ptr, items.data(), sizeof(BatchItem) * items.size(), cudaMemcpyHostToDevice,
                           b->stream),
           "upload");
    int dev = 0, sms = 0;
    CK(cudaGetDevice(&dev), "device");
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "device");
    b->only_direct = std::all_of(dirs.begin(), dirs.end(), [](int d) { return d != 0; });
    const int per_sm = sim_batch_ctas_per_sm(threads, smem, b->only_direct);
    if (per_sm < 1) return fail(TVBX_E_UNSUPPORTED, "batch kernel does not fit %d threads / %zu bytes", threads, smem);
    b->grid = (int32_t)std::max<int64_t>(1, std::min<int64_t>((int64_t)sms * per_sm, (int64_t)items.size()));
    b->threads = threads;
    b->smem_budget = budget;
    b->direct = direct;
    CK(cudaStreamSynchronize(b->stream), "batch upload");

    // capture the device work of one run
    CK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal), "graph capture");
    cudaError_t ce = cudaSuccess;
    tvbx_status fst = TVBX_OK;
    int64_t kernels = 0;
    for (size_t j = 0; j < nj && ce == cudaSuccess; ++j) {
        tvbx_sweep* h = b->jobs[j];
        const SimArgs& a = jobs[j].a;   // round 0
        if ((ce = cudaMemsetAsync(h->d_error.ptr, 0, sizeof(uint32_t), b->stream)) != cudaSuccess) break;
        if ((ce = launch_init_state(a, b->stream)) != cudaSuccess) break;
        ++kernels;
        for (const GroupDev& g : plans[j].gdev) {
            if ((ce = launch_init_ring(g.ring, (int64_t)g.H * h->N * g.stride, a.m.E0, b->stream)) != cudaSuccess) break;
            ++kernels;
        }
        if (ce != cudaSuccess) break;
        if (ou_off[j] >= 0) {   // the job's whole OU table
            if ((ce = cudaMemsetAsync(h->d_ou_state.ptr, 0, sizeof(float) * h->N, b->stream)) != cudaSuccess) break;
            if ((ce = launch_ou_table(a.m, b->d_ou.as<float>() + ou_off[j], h->d_ou_state.as<float>(), h->N, 0,
                                      (int32_t)run_cfgs[j].n_steps, a.seed, b->stream)) != cudaSuccess)
                break;
            ++kernels;
        }
        if (run_cfgs[j].series_mode == TVBX_SERIES_STREAM)
            ce = cudaMemsetAsync(h->d_fcacc.ptr, 0, sizeof(float) * (size_t)h->P * ((size_t)h->N * h->N + h->N),
                                 b->stream);
    }
    if (ce == cudaSuccess) ce = cudaMemsetAsync(b->d_head.ptr, 0, sizeof(int32_t) * (size_t)R, b->stream);
    std::vector<char> shift_set(nj, 0);
    for (int64_t r = 0; r < R && ce == cudaSuccess && fst == TVBX_OK; ++r) {
        const int64_t n_r = item_off[(size_t)r + 1] - item_off[(size_t)r];
        if (n_r > 0) {
            const int32_t grid_r = (int32_t)std::max<int64_t>(1, std::min<int64_t>((int64_t)sms * per_sm, n_r));
            ce = launch_sim_batch(b->d_jobs.as<BatchJob>(), b->d_items.as<BatchItem>() + item_off[(size_t)r],
                                  (int32_t)n_r, b->d_head.as<int32_t>() + r, grid_r, threads, smem, b->only_direct,
                                  b->stream);
            ++kernels;
        }
        for (size_t j = 0; j < nj && ce == cudaSuccess && fst == TVBX_OK; ++j) {
            const SimArgs& a = jobs[(size_t)r * nj + j].a;
            if (run_cfgs[j].series_mode != TVBX_SERIES_STREAM || a.n_chunk <= 0) continue;
            bool ss = shift_set[j] != 0;
            kernels += ss ? 2 : 3;   // (shift,) moments, accumulation
            fst = stream_fc_chunk(b->jobs[j], a, a.n0, a.n_chunk, ss, b->stream);
            shift_set[j] = ss ? 1 : 0;
        }
    }
    cudaGraph_t g = nullptr;
    cudaError_t ee = cudaStreamEndCapture(b->stream, &g);
    if (ce != cudaSuccess || ee != cudaSuccess || fst != TVBX_OK) {
        if (g) cudaGraphDestroy(g);
        (void)cudaGetLastError();
        if (fst != TVBX_OK && ce == cudaSuccess && ee == cudaSuccess) return fst;
        return cuda_fail(ce != cudaSuccess ? ce : ee, "batch graph capture");
    }
    b->graph = g;
    CK(cudaGraphInstantiate(&b->exec, g, 0), "batch graph instantiate");
    size_t nodes = 0;
    CK(cudaGraphGetNodes(g, nullptr, &nodes), "batch graph");
    b->graph_nodes = (int64_t)nodes;
    b->graph_kernels = kernels;
    b->cfgs_run = run_cfgs;
    b->gens.resize(nj);
    for (size_t j = 0; j < nj; ++j) b->gens[j] = b->jobs[j]->gen;
    b->built = true;
    return TVBX_OK;
}

}  // namespace

extern "C" {

tvbx_status tvbx_batch_create(tvbx_sweep* const* jobs, const tvbx_run_cfg* cfgs, int32_t n_jobs, tvbx_batch** out)
{
    if (!jobs || !cfgs || !out || n_jobs < 1) return fail(TVBX_E_INVALID_ARG, "need jobs, cfgs, out and n_jobs >= 1");
    *out = nullptr;
    for (int32_t j = 0; j < n_jobs; ++j) {
        if (!jobs[j]) return fail(TVBX_E_INVALID_ARG, "job %d: NULL handle", j);
        for (int32_t i = 0; i < j; ++i)
            if (jobs[i] == jobs[j]) return fail(TVBX_E_INVALID_ARG, "job %d repeats job %d", j, i);
        const tvbx_run_cfg& c = cfgs[j];
        if (!(c.dt_ms > 0.0) || c.tavg_steps < 1 || c.n_steps < 1 || c.n_steps > INT32_MAX)
            return fail(TVBX_E_INVALID_ARG, "job %d: need dt_ms > 0, tavg_steps >= 1, 1 <= n_steps < 2^31", j);
        if (c.withhold_step != 0) return fail(TVBX_E_INVALID_ARG, "job %d: withhold_step is not used by batches", j);
    }
    auto* b = new tvbx_batch;
    b->jobs.assign(jobs, jobs + n_jobs);
    b->cfgs.assign(cfgs, cfgs + n_jobs);
    cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        delete b;
        return cuda_fail(e, "batch stream");
    }
    *out = b;
    return TVBX_OK;
}

tvbx_status tvbx_batch_tune(tvbx_batch* b, int64_t trial_steps, int32_t* threads_out, int32_t* smem_kb_out,
                            float* trial_ms, int32_t* n_trials)
{
    if (!b) return fail(TVBX_E_INVALID_ARG, "NULL batch");
    if (trial_steps < 1) return fail(TVBX_E_INVALID_ARG, "trial_steps must be >= 1");
    // general body under shared-memory budgets, and register tiles (general
    // body only for jobs with more regions than threads)
    struct Cand { int32_t threads; size_t budget; bool direct; };
    const Cand cands[] = {{256, 100 * 1024, false}, {512, 100 * 1024, false}, {256, 200 * 1024, false},
                          {512, 200 * 1024, false}, {128, 64 * 1024, false},  {256, 64 * 1024, false},
                          {512, 200 * 1024, true},  {768, 200 * 1024, true}};
    float best = INFINITY;
    Cand win{0, 0, false};
    int32_t k = 0;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0), "event");
    CK(cudaEventCreate(&e1), "event");
    for (const Cand& c : cands) {
        float ms = INFINITY;
        if (batch_build(b, c.threads, c.budget, trial_steps, c.direct) == TVBX_OK) {
            cudaError_t e = cudaGraphLaunch(b->exec, b->stream);   // warm-up
            if (e == cudaSuccess) e = cudaEventRecord(e0, b->stream);
            if (e == cudaSuccess) e = cudaGraphLaunch(b->exec, b->stream);
            if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e != cudaSuccess) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                return cuda_fail(e, "batch trial");
            }
            note_launch(2 * b->graph_kernels);
        } else {
            (void)cudaGetLastError();
        }
        if (trial_ms) trial_ms[k] = ms;
        ++k;
        if (ms < best) { best = ms; win = c; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!(best < INFINITY)) return fail(TVBX_E_UNSUPPORTED, "no batch configuration fits every job");
    if (n_trials) *n_trials = k;
    tvbx_status st = batch_build(b, win.threads, win.budget, 0, win.direct);
    if (st != TVBX_OK) return st;
    if (threads_out) *threads_out = win.threads;
    if (smem_kb_out) *smem_kb_out = (int32_t)(win.budget / 1024);
    return TVBX_OK;
}

tvbx_status tvbx_batch_run(tvbx_batch* b)
{
    if (!b) return fail(TVBX_E_INVALID_ARG, "NULL batch");
    if (tvbx_status st = batch_adopt_jobs(b)) return st;
    bool stale = !b->built;
    for (size_t j = 0; j < b->jobs.size() && !stale; ++j) stale = b->jobs[j]->gen != b->gens[j];
    for (size_t j = 0; j < b->jobs.size() && !stale; ++j) stale = b->cfgs_run[j].n_steps != b->cfgs[j].n_steps;
    if (stale) {
        tvbx_status st = batch_build(b, b->threads, b->smem_budget, 0, b->direct);
        if (st != TVBX_OK) return st;
    }
    CK(cudaGraphLaunch(b->exec, b->stream), "batch launch");
    note_launch(b->graph_kernels);
    for (size_t j = 0; j < b->jobs.size(); ++j) {
        b->jobs[j]->stream = b->stream;
        finish_run(b->jobs[j], b->cfgs_run[j]);
    }
    CK(cudaStreamSynchronize(b->stream), "batch run");
    return TVBX_OK;
}

tvbx_status tvbx_batch_info(const tvbx_batch* b, int32_t* threads, int32_t* smem_kb, int64_t* n_items, int32_t* grid,
                            int64_t* graph_nodes)
{
    if (!b) return fail(TVBX_E_INVALID_ARG, "NULL batch");
    if (threads) *threads = b->threads;
    if (smem_kb) *smem_kb = (int32_t)(b->smem_budget / 1024);
    if (n_items) *n_items = b->n_items;
    if (grid) *grid = b->grid;
    if (graph_nodes) *graph_nodes = b->graph_nodes;
    return TVBX_OK;
}

tvbx_status tvbx_batch_destroy(tvbx_batch* b)
{
    if (!b) return TVBX_OK;
    if (b->stream) cudaStreamSynchronize(b->stream);
    // the jobs ran on the batch's stream: hand them back to the default
    // stream before that stream is destroyed
    for (tvbx_sweep* h : b->jobs)
        if (h->stream == b->stream) h->stream = nullptr;
    delete b;
    return TVBX_OK;
}

}  // extern "C"

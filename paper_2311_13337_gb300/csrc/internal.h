// Engine-internal declarations shared by the tvbx CUDA translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "tvbx.h"

namespace tvbx {

// Process-wide count of kernel launches made by this library.
void note_launch(uint64_t n = 1);

// Record the message of a failing call (returned by tvbx_last_error) and
// return `code`.
tvbx_status report_error(tvbx_status code, const char* fmt, ...);

// Number of per-(set, region) state words kept across steps and chunks:
// E, I, C_ee, C_ei, C_ii, W_e, W_i, OU, then the temporal-average accumulators
// of E and I, then compensated running sums (sum, carry) of the E and I
// samples, then the carries of the compensated Euler updates of W_e and W_i.
enum {
    SV_E = 0, SV_I, SV_CEE, SV_CEI, SV_CII, SV_WE, SV_WI, SV_OU,
    SV_ACC_E, SV_ACC_I, SV_SUM_E, SV_CMP_E, SV_SUM_I, SV_CMP_I, SV_CWE, SV_CWI, SV_COUNT
};

// Model constants prepared for the device (FP32, with derived quantities).
struct DevModel {
    float g_L, C_m, E_e, E_i;
    float qe, qi;            // Q_e tau_e, Q_i tau_i (nS ms)
    float tau_e, tau_i;
    float K_e, K_i;
    float inv_Ne, inv_Ni, inv_T;
    float P_e[10], P_i[10];
    float mu0, inv_dmu0, sig0, inv_dsig0, tau0, inv_dtau0;
    float gL_over_Cm;
    float rate_floor;
    float b_i, a_i, inv_tau_w_i;
    float E_min, E_max;
    float E0, I0;
    float C_div;             // |covariance| above this marks the set diverged
    // OU (Eq. 4) by Euler-Maruyama: OU' = OU + ou_a (mu - OU) + ou_b xi
    float ou_a, ou_b, ou_mu;
    float dt;
    // Reduced transfer function (model_device.cuh), used when tau_e == tau_i
    int32_t reduced;         // 1: tau_e == tau_i
    float tau;               // the common synaptic time constant
    float ke, ki;            // qe^2, qi^2
    float dE;                // E_e - E_i
    float be, bi;            // qi dE, -qe dE
    float two_be, two_bi;
    float gLEe;              // g_L E_e
    float v0, v1, v1qe, v1qi, v1be, two_v1;   // V = v0 - v1 a_e / mu_G
    float s0, s1, s1h, s1q;  // S = s1 sigma_V - s0, s1 / 2, s1 / 4
    float z0, z1, z1sq, two_z1;               // Z = z0 + z1 / mu_G
    float sq_e, sq_i;        // 2 ke be^2, 2 ki bi^2
    float cp_e[10], cp_i[10];  // (V_thre - mu_V) / sqrt(2) as a polynomial in (V, S, Z)
};

// One speed group: sets sharing a delay matrix and a ring buffer.
struct GroupDev {
    float* ring;               // [H][N][P_g], E of the group's sets
    const int32_t* row_ptr;    // [N + 1] CSR rows of the nonzero weights u_kj; each row
                               // starts at an index of the parity of k (padded with a
                               // zero-weight self entry of delay 1) and ends with its
                               // zero-delay entries
    const int32_t* row_mid;    // [N] first zero-delay entry of each row
    const uint32_t* col_dly;   // [nnz] (delay << 16) | j
    const float* w;            // [nnz] u_kj
    int32_t H;                 // ring depth (max delay + 2)
    int32_t P_g;               // sets in the group
    int32_t p_base;            // first internal set index of the group
    int32_t stride;            // ring row stride in floats (P_g rounded up to 32)
    int32_t nnz;               // CSR entries (nonzero weights and padding)
    int32_t nnz_d;             // entries with a delay of at least one step
};

// Device error word bits (SimArgs::error).
constexpr uint32_t TVBX_DEVERR_TIMEOUT = 1u;   // a bounded wait gave up

// One CTA's work: sets [q0, q0 + nq) of group g (q relative to the group).
struct TileDev {
    int32_t group;
    int32_t q0;
    int32_t nq;
    int32_t pad;
};

// Arguments of one simulation chunk launch.
// Layout of a rate series: element (sample t, region k, set p) at
//   (p / 4) sg + t st + k sk + p % 4.
// [T][N][P] (sets fastest; the external layout): sg = 4, st = N P, sk = P.
// Set-blocked [ceil(P / 4)][T_buf][N][4] (the engine's own series): sg = 4 N
// T_buf, st = 4 N, sk = 4 -- the 16 bytes of a group of 4 sets for all
// regions of a sample are contiguous, so readers that own a group of sets
// read whole lines along the regions.
struct SeriesLayout {
    int64_t sg, st, sk;
};
__host__ __device__ __forceinline__ int64_t series_index(const SeriesLayout& l, int64_t t, int64_t k, int64_t p)
{
    return (p >> 2) * l.sg + t * l.st + k * l.sk + (p & 3);
}
inline SeriesLayout layout_tnp(int64_t N, int64_t P) { return SeriesLayout{4, N * P, P}; }
inline SeriesLayout layout_blocked(int64_t N, int64_t T_buf) { return SeriesLayout{4 * N * T_buf, 4 * N, 4}; }

struct SimArgs {
    DevModel m;
    const GroupDev* groups;
    const TileDev* tiles;
    const float* prm;          // [TVBX_N_AXES][P] per-set parameters (internal order)
    const int64_t* ext_index;  // [P] external set index (keys per-set noise)
    float* state;              // [SV_COUNT][N][P]
    float* series;             // E samples, layout sl
    SeriesLayout sl;           // of series and series_i
    const float* ou_table;     // [n_chunk][N] shared OU values, or null
    uint32_t* status;          // [P]
    uint32_t* error;           // device error word (TVBX_DEVERR_*)
    int64_t withhold_step;     // step whose bulk copies are withheld (-1: none; testing)
    uint32_t wait_limit;       // try_wait attempts before a wait gives up
    int64_t n0;                // global index of the chunk's first step
    int32_t n_chunk;           // steps in this chunk
    int32_t N;                 // regions
    int32_t P;                 // sets (internal)
    int32_t ts;                // steps per sample
    int64_t T;                 // samples in the run
    int32_t transient;         // samples excluded from the running sums
    int32_t noise_per_set;
    uint64_t seed;
    int64_t p_offset;
    float* series_i;           // I samples (layout sl), or null
};

// Kernels / launchers (sim.cu).
cudaError_t launch_init_state(const SimArgs& a, cudaStream_t s);
cudaError_t launch_init_ring(float* ring, int64_t count, float value, cudaStream_t s);
cudaError_t launch_ou_table(const DevModel& m, float* table, float* ou_state, int32_t N,
                            int64_t n0, int32_t n_chunk, uint64_t seed, cudaStream_t s);
cudaError_t launch_sim_chunk(const SimArgs& a, int32_t n_tiles, int32_t pb, cudaStream_t s);
cudaError_t launch_tf_eval(const DevModel& m, int pop, int64_t n, const float* x_e, const float* x_i,
                           const float* W, const float* E_L, const float* C, float* out, cudaStream_t s);
// Prefetching kernel (sim_fast.cu): variant 0 = 16 sets per CTA, 1 = 32.
cudaError_t launch_sim_fast(const SimArgs& a, int variant, int32_t n_tiles, int nnz_max, cudaStream_t s);
bool sim_fast_fits(int variant, int N, int nnz_max);
int sim_fast_pb(int variant);
bool sim_fast_packed(int variant);   // FP32x2 kernel (needs tau_e == tau_i)
int sim_fast_variants();
size_t sim_fast_smem_bytes(int variant, int N, int nnz);
int sim_threads(int N, int pb);
size_t sim_smem_bytes(int N, int pb);

// FC (fc.cu).
// One job of a batch (device): its SimArgs cover all steps (n0 = 0,
// n_chunk = n_steps, OU table for every step); pb = its tile width.
struct BatchJob {
    SimArgs a;
    int32_t pb;       // tile width of the job
    int32_t direct;   // 1: register-tile body (N pb / 4 <= blockDim), 0: general body
};
struct BatchItem {
    int32_t job, tile;
};
// Register-tile kernel for large connectomes: tile width for N regions (0 if
// N is too large), and the launch of one chunk.
int sim_direct_pb(int N);
cudaError_t launch_sim_direct(const SimArgs& a, int32_t n_tiles, int32_t pb, cudaStream_t s);
cudaError_t launch_sim_batch(const BatchJob* jobs, const BatchItem* items, int32_t n_items, int32_t* head,
                             int32_t grid, int32_t threads, size_t smem, bool only_direct, cudaStream_t s);
int sim_batch_ctas_per_sm(int32_t threads, size_t smem, bool only_direct);

struct FcArgs {
    const float* series;       // samples, layout sl
    SeriesLayout sl;
    const float* state;        // [SV_COUNT][N][P] (running sums give the shift)
    int32_t N, P;
    int64_t t_begin, t_end;    // samples used: [t_begin, t_end)
    int32_t blk;               // samples per FCD block (0: one block)
    int32_t n_blocks;
    float* blocks;             // [P][n_blocks][N*N + N] block moments (nullable)
    float* fc;                 // [P][N][N] internal order (nullable)
    float* chi;                // [P]
    float* mean_fc;            // [P]
    uint32_t* status;          // [P]
    const float* shift;        // [N][P] shift m_k when state is NULL (nullable: 0)
    uint32_t* error;           // device error word (tensor-core path)
    uint32_t wait_limit;       // try_wait attempts before a wait gives up
};
// Block moments (SIMT, FP32 CUDA-core FMAs).
cudaError_t launch_fc_moments(const FcArgs& a, cudaStream_t s);
// From the block moments: Pearson FC, chi, mean FC and (nw > 0) the FCD over
// nw windows of m blocks of Lw samples, in one kernel when its shared memory
// fits; vec_scratch ([P][nw][N(N-1)/2]) is used only when it does not.
cudaError_t launch_fc_reduce(const FcArgs& a, int32_t m, int32_t nw, int64_t Lw, float* vec_scratch, float* fcd,
                             cudaStream_t s);
size_t fc_reduce_needs_vec_scratch(int N, int nb, int nw);
// Tensor-core block moments (precision TVBX_FC_BF16 .. TVBX_FC_TF32X3);
// N <= 128.
cudaError_t launch_fc_tc_moments(const FcArgs& a, int prec, cudaStream_t s);
bool fc_tc_supported(int N, int prec);
// Pearson FC, chi and mean FC from the block moments.
cudaError_t launch_fc_finalize(const FcArgs& a, cudaStream_t s);
// Shift m_k = mean of up to 64 evenly spaced samples (standalone series).
cudaError_t launch_fc_accumulate(const float* add, float* acc, int64_t n, cudaStream_t s);
cudaError_t launch_fc_shift(const float* series, const SeriesLayout& sl, int32_t N, int64_t P, int64_t t_begin,
                            int64_t t_end, float* shift, cudaStream_t s);
cudaError_t launch_fcd(const float* blocks, int32_t P, int32_t N, int32_t n_blocks,
                       int32_t blocks_per_window, int32_t n_windows, int64_t window_samples,
                       float* vec_scratch, float* fcd, cudaStream_t s);
cudaError_t launch_summary(const float* state, int32_t N, int32_t P, int64_t n_samples,
                           float* mean_e_hz, float* mean_i_hz, cudaStream_t s);

}  // namespace tvbx

/*
 * tvbx — GB300 (sm_103a) engine for the data-parallel hot path of the
 * TVB-AdEx parameter-space exploration of arXiv 2311.13337 ("Vast TVB
 * parameter space exploration"): lock-step time integration of many
 * independent whole-brain AdEx mean-field simulations, one per parameter
 * point, and the reduction of their excitatory-rate series to functional
 * connectivity (FC), FC dynamics (FCD) and per-set summaries.
 *
 * Conventions for every entry point:
 *   - Return value: TVBX_OK (0) or a negative tvbx_status. The message of the
 *     last failure on the calling thread is returned by tvbx_last_error().
 *   - Units: time ms, rates kHz inside the model (Hz where a name says _hz),
 *     voltages mV, conductances nS, capacitance pF, currents pA, tract
 *     lengths mm, conduction speed m/s (= mm/ms).
 *   - Inputs passed by pointer are copied before the call returns; the caller
 *     keeps ownership. Outputs go to caller-owned buffers whose memory kind is
 *     given by a `mem` argument (TVBX_MEM_HOST or TVBX_MEM_DEVICE). Host output
 *     calls synchronise the handle's stream before returning.
 *   - Set order: parameter sets are numbered in grid order (Cartesian product,
 *     last axis fastest) or in the order of an explicit point list. All per-set
 *     outputs use that order.
 *   - A handle is used by one host thread at a time; device work is enqueued
 *     on the stream passed to tvbx_run (or the default stream when NULL).
 *   - No entry point falls back to a CPU path: without a usable CUDA device
 *     they return TVBX_E_CUDA.
 */
#ifndef TVBX_H
#define TVBX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t tvbx_status;
#define TVBX_OK             0
#define TVBX_E_INVALID_ARG (-1) /* bad pointer, size, range or combination */
#define TVBX_E_OOM         (-2) /* device allocation failed (P x H x N too large) */
#define TVBX_E_CUDA        (-3) /* CUDA runtime or launch error, or no device */
#define TVBX_E_NUMERIC     (-4) /* every set became non-finite */
#define TVBX_E_TIMEOUT     (-5) /* a bounded device-side wait gave up (reported by the
                                   first output call after the run) */
#define TVBX_E_BAD_STATE   (-6) /* call out of order (e.g. tvbx_fc before tvbx_run) */
#define TVBX_E_UNSUPPORTED (-7) /* valid request this build does not implement */

#define TVBX_MEM_HOST   0
#define TVBX_MEM_DEVICE 1

/* Per-set status bits (tvbx_summary). */
#define TVBX_SET_NONFINITE 1u /* a state variable became NaN or Inf */
#define TVBX_SET_CLAMP_HI  2u /* E or I was clamped at the upper bound */
#define TVBX_SET_CLAMP_LO  4u /* E or I was clamped at the lower bound */
#define TVBX_SET_ZERO_VAR  8u /* a region's E series had zero variance (FC row 0) */
#define TVBX_SET_DIVERGED 16u /* a covariance passed C_div: the second-order
                                 moment closure broke down (dynamics unaltered) */

/* Sweepable axes: the per-set parameters of the sweep (Sec. "Vast parameter
 * space exploration and analysis", Table 4, plus the leak reversals of
 * Table 3). */
enum tvbx_axis {
    TVBX_AXIS_G = 0,     /* global coupling g (Eq. 5), dimensionless */
    TVBX_AXIS_B_E,       /* spike-frequency adaptation b_e (Eq. 3), pA */
    TVBX_AXIS_TAU_W_E,   /* adaptation time constant tau_w,e (Eq. 3), ms */
    TVBX_AXIS_E_L_E,     /* leak reversal of the excitatory population, mV */
    TVBX_AXIS_E_L_I,     /* leak reversal of the inhibitory population, mV */
    TVBX_AXIS_SPEED,     /* conduction speed (delays = length / speed), m/s */
    TVBX_AXIS_A_E,       /* subthreshold adaptation a_e (Eq. 3), nS */
    TVBX_AXIS_W_NOISE,   /* weight of the OU noise in the excitatory input (Eq. 5) */
    TVBX_AXIS_CF_EE,     /* constant input c_F{e,e} (Eq. 5), kHz */
    TVBX_AXIS_CF_EI,     /* c_F{e,i}, kHz */
    TVBX_AXIS_CF_IE,     /* c_F{i,e}, kHz */
    TVBX_AXIS_CF_II,     /* c_F{i,i}, kHz */
    TVBX_N_AXES
};

/* Model constants shared by all sets of a sweep. The transfer function is
 * the semi-analytic template the paper cites (Sec. "Transfer Function",
 * Eq. 5) with the threshold polynomial of Table 1; the rate, covariance and
 * adaptation equations are Eq. 1-3 and the noise is Eq. 4. */
typedef struct {
    double g_L, C_m, E_e, E_i, Q_e, Q_i, tau_e, tau_i;
    double K_e, K_i;          /* synaptic inputs per cell from the e / i pools */
    double N_e, N_i;          /* population sizes in the finite-size term of Eq. 2 */
    double T;                 /* time constant of Eq. 1-2, ms */
    double P_e[10], P_i[10];  /* Table 1 rows (RS for e, FS for i), mV, in the
                                 table's column order */
    double mu0, dmu0, sig0, dsig0, tau0, dtau0; /* normalisation of mu_V, sigma_V, tau_V^N */
    double rate_floor;        /* added to K*nu so that sigma_V > 0, kHz */
    double tau_OU, mu_OU, sigma_OU; /* Eq. 4 */
    double b_i, a_i, tau_w_i; /* inhibitory adaptation */
    double E_min, E_max;      /* E and I are clamped to [E_min, E_max] after each step, kHz */
    double E0, I0;            /* initial rates, kHz; also the constant prehistory of E */
    double C_div;             /* |covariance| above this sets TVBX_SET_DIVERGED, kHz^2 */
    double defaults[TVBX_N_AXES]; /* value of each axis when it is not swept */
} tvbx_model;

/* One swept axis: n values, either values[0..n-1] or, when values is NULL,
 * n equally spaced values in [lo, hi] with both ends included (Sec. "TVB-AdEx
 * to GPU": "-s0 6 generates six values equally spaced within the defined
 * range"). */
typedef struct {
    int32_t axis;             /* enum tvbx_axis */
    int32_t n;                /* >= 1 */
    double lo, hi;
    const double* values;     /* nullable, host memory, n entries */
} tvbx_axis_spec;

/* Cartesian product of the axes, last axis fastest: the work items. */
typedef struct {
    int32_t n_axes;
    const tvbx_axis_spec* axes;
} tvbx_grid;

typedef struct tvbx_sweep tvbx_sweep;

/* Integration settings (Sec. "TVB-AdEx to GPU" and "MPI", last paragraph:
 * forward Euler; Sec. "Output": the observable is the mean of the inner
 * steps). */
typedef struct {
    double dt_ms;             /* Euler step, ms (> 0) */
    int64_t n_steps;          /* steps to integrate from the initial state (>= 0) */
    int32_t tavg_steps;       /* steps per temporal-average sample (>= 1) */
    int32_t noise_per_set;    /* 0: one OU process per region, shared by all
                                 sets (the paper's precomputed noise);
                                 1: an independent process per set and region */
    uint64_t seed;            /* Philox4x32-10 key */
    int64_t p_offset;         /* global index of set 0; keys per-set noise so
                                 that shards of a sweep reproduce it exactly */
    int32_t transient_samples;/* samples excluded from means, FC, chi */
    int32_t chunk_steps;      /* steps per kernel launch; 0 = automatic. Must be
                                 a multiple of tavg_steps when given. */
    int32_t kernel;           /* TVBX_KERNEL_AUTO, TVBX_KERNEL_GENERAL, or
                                 TVBX_KERNEL_PREFETCH + v for prefetch variant v */
    int32_t withhold_step;    /* testing the failure path: 0 = off; s > 0 makes the
                                 TMA-copy kernels withhold the copies of step s - 1
                                 and shorten their wait, so the wait expires and the
                                 run reports TVBX_E_TIMEOUT (no fault, the context
                                 stays usable). Other kernels ignore it. */
    int32_t series_mode;      /* TVBX_SERIES_KEEP (0) or TVBX_SERIES_STREAM */
    int32_t keep_i_series;    /* 1: also keep the inhibitory rate series
                                 [T][N][P] (block means like E; read with
                                 tvbx_series_pop_range, pop 1), e.g. for the
                                 PLI of the I rates (Table 2 PLI_i) through
                                 tvbx_series_analysis; needs TVBX_SERIES_KEEP
                                 and doubles the series memory. 0: E only. */
} tvbx_run_cfg;

/* Series modes of tvbx_run_cfg.
 * TVBX_SERIES_KEEP: the whole E series [T][N][P] stays on the device.
 * TVBX_SERIES_STREAM: only one chunk of samples is kept (chunk_steps, or the
 *   automatic chunk of about 5,000 steps, divided by tavg_steps). After each
 *   chunk the library folds its samples after the transient into per-set FC
 *   moments (Eq. 6: sums of x_k and x_k x_j about a fixed shift, the mean of
 *   up to 64 samples of the first chunk after the transient; FP32 CUDA-core
 *   products, summed over chunks in FP32), so the series memory no longer
 *   grows with the duration. tvbx_fc then returns FC, chi and mean FC from the
 *   moments (any precision argument; fcd_window must be 0: the FCD needs the
 *   whole series), and tvbx_series / tvbx_series_range return
 *   TVBX_E_BAD_STATE. Needs n_regions <= 384. Means, status and the final
 *   state are those of TVBX_SERIES_KEEP, bit for bit. */
#define TVBX_SERIES_KEEP 0
#define TVBX_SERIES_STREAM 1
#define TVBX_KERNEL_AUTO     0 /* fastest kernel that fits the sweep */
#define TVBX_KERNEL_DIRECT 100 /* register tiles for connectomes too large for the
                                  prefetch buffer (up to 768 regions): 4 sets of
                                  one region per thread, 16-byte ring gathers;
                                  results bit-identical to TVBX_KERNEL_GENERAL */
#define TVBX_KERNEL_GENERAL  1 /* any size: state in shared memory, direct gathers */
#define TVBX_KERNEL_PREFETCH 2 /* + v: next-step gather prefetched into shared
                                  memory; CTA of 16 or 32 sets; cp.async into one
                                  buffer: v = 0: 16 sets, 2 sets x 1 region per
                                  thread; 1: 32 sets, 4 x 1; 2: 16 sets, 1 x 2;
                                  3: 16 sets, 2 x 2; TMA bulk copies into two
                                  buffers: 4: 16 sets, 2 x 1; 5: 16 sets, 1 x 2;
                                  cp.async, 8 sets, two CTAs per SM: 6: 2 x 1;
                                  7: 1 x 2; two sets per thread in packed
                                  FP32x2 arithmetic, TMA bulk copies into two
                                  buffers (only for tau_e == tau_i, else
                                  TVBX_E_UNSUPPORTED): 8: 12 sets, 2 x 1;
                                  9: 16 sets, 2 x 1; 10: 8 sets, 2 x 1;
                                  11: 16 sets, 2 x 2; TMA bulk copies into
                                  one buffer, one CTA barrier per step:
                                  12: 32 sets, 4 x 1; 13: 16 sets, 2 x 1;
                                  14: 32 sets, 2 x 2; cp.async into two
                                  buffers, one barrier per step: 15: 16
                                  sets, 2 x 1; 16: 16 sets, 1 x 2 */

/* FC settings (Sec. "Output": FC from the covariance of the series,
 * Eq. 6 Pearson; FCD over sliding windows). */
typedef struct {
    int32_t precision;        /* one of TVBX_FC_* below */
    int32_t fcd_window;       /* samples per FCD window; 0 = no FCD */
    int32_t fcd_step;         /* samples between window starts; fcd_window must
                                 be a multiple of fcd_step */
    int32_t series_layout;    /* tvbx_fc_series only: TVBX_LAYOUT_TNP (0) or
                                 TVBX_LAYOUT_SET4 (below); tvbx_fc reads the
                                 sweep's own series and ignores it */
} tvbx_fc_cfg;

/* Layouts of a series given to tvbx_fc_series.
 * TVBX_LAYOUT_TNP: [n_samples][n_regions][n_sets], sets fastest.
 * TVBX_LAYOUT_SET4: groups of 4 sets, [ceil(n_sets / 4)][n_samples][n_regions][4]
 *   (element (t, k, p) at ((p / 4) n_samples + t) n_regions 4 + 4 k + p % 4;
 *   the last group padded to 4 sets, padding never read). The engine keeps its
 *   own series this way: the FC readers then load whole lines along the
 *   regions. */
#define TVBX_LAYOUT_TNP 0
#define TVBX_LAYOUT_SET4 1
/* The Gram matrix G = Z Z^T of the shifted series Z (the contraction behind
 * the covariance of Eq. 6) is formed
 *   FP32:    with FP32 CUDA-core FMAs;
 *   BF16:    on the tensor cores from Z rounded to BF16, FP32 accumulation;
 *   BF16X3:  split precision, Z = H + L with H, L in BF16, G = H H^T + H L^T
 *            + L H^T (three MMAs per K step; symmetric up to the FP32
 *            accumulation), FP32 accumulation;
 *   TF32, TF32X3: the same with TF32 operands.
 * The tensor-core forms need n_regions <= 112. The row sums of Z use
 * compensated FP32 summation in the tensor-core forms and plain FP32 sums in
 * the FP32 form (the shifted rows sum to near zero, so either error is far
 * below that of the Gram matrix). */
#define TVBX_FC_FP32   0
#define TVBX_FC_BF16   1
#define TVBX_FC_BF16X3 2
#define TVBX_FC_TF32   3
#define TVBX_FC_TF32X3 4

/* Library version string. */
const char* tvbx_version(void);

/* Message of the last failed call on this thread ("" if none). Valid until
 * the next failing call on the same thread. */
const char* tvbx_last_error(void);

/* Device memory of the handles (sweeps, batches, surrogates; no counterpart
 * in the paper). By default it comes from cudaMalloc / cudaFree.
 * tvbx_set_allocator installs a caller's pair instead, for example a
 * framework's caching allocator so that the engine and the framework share
 * one pool. The pair is process-wide and serves allocations made after the
 * call; each buffer is released through the pair that allocated it, after a
 * device synchronisation (a caching allocator may hand a freed block out at
 * once while queued work still uses it). alloc(bytes, ctx) returns a device
 * pointer aligned to at least 256 bytes, or NULL on failure (reported as
 * TVBX_E_OOM); free(ptr, ctx) releases it. Both NULL restore the default.
 * The scratch of the stateless calls (tvbx_fc_series, tvbx_series_analysis,
 * tvbx_phfcd, tvbx_fc_fitness, tvbx_top_k) comes from CUDA's stream-ordered
 * allocator, tvbx_cell_rates uses cudaMalloc for its call, and
 * tvbx_fc_noalloc allocates nothing. Errors: TVBX_E_INVALID_ARG when only one
 * of the pair is given. */
typedef void* (*tvbx_alloc_fn)(uint64_t bytes, void* ctx);
typedef void (*tvbx_free_fn)(void* ptr, void* ctx);
tvbx_status tvbx_set_allocator(tvbx_alloc_fn alloc, tvbx_free_fn free_fn, void* ctx);

/* Fill *out with the engine's default model constants and axis defaults.
 * Needs no GPU. */
tvbx_status tvbx_model_defaults(tvbx_model* out);

/* Create a sweep over a grid of parameter sets.
 *   weights    [n_regions][n_regions] row-major connectome weights u_kj
 *              (Eq. 5: region k receives sum_j u_kj nu_e,j(t - tau_kj)); host.
 *   tract_mm   [n_regions][n_regions] tract lengths in mm (delays tau_kj =
 *              length / speed, Eq. 5); host, >= 0.
 *   grid       the swept axes; an empty grid gives one set at the defaults.
 *   model      constants; NULL = tvbx_model_defaults().
 *   out        receives the handle (release with tvbx_sweep_destroy).
 * Errors: TVBX_E_INVALID_ARG for NULL pointers, n_regions < 1, non-finite or
 * negative lengths, unknown or repeated axes, n < 1; TVBX_E_CUDA without a
 * device. Device memory is allocated by tvbx_run, not here. */
tvbx_status tvbx_sweep_create(const double* weights, const double* tract_mm, int32_t n_regions,
                              const tvbx_grid* grid, const tvbx_model* model, tvbx_sweep** out);

/* Create a sweep over explicit points: params[n_sets][TVBX_N_AXES] (host),
 * one row per set in enum tvbx_axis order. Otherwise as tvbx_sweep_create. */
tvbx_status tvbx_sweep_create_points(const double* weights, const double* tract_mm,
                                     int32_t n_regions, int64_t n_sets, const double* params,
                                     const tvbx_model* model, tvbx_sweep** out);

/* Number of sets, regions and (after tvbx_run) samples per region. */
tvbx_status tvbx_sweep_info(const tvbx_sweep* h, int64_t* n_sets, int32_t* n_regions,
                            int64_t* n_samples);

/* Integrate every set for cfg->n_steps steps from the initial state
 * (Eq. 1-5, forward Euler; delays rint(length / (speed dt)), ties to even;
 * constant prehistory E0). Each step, for every (set, region): gather the
 * delayed coupling from the set's ring buffer, evaluate both transfer
 * functions with their gradients and Hessians, advance E, I, C_ee, C_ei,
 * C_ii, W_e, W_i and OU, clamp E and I, write E to the ring, and accumulate
 * the temporal average. The work is enqueued on `cuda_stream` (a
 * cudaStream_t; NULL = default stream) and the call returns without waiting.
 * Allocates (or reuses) the ring buffers [H][N][P_group], the state, and the
 * E series [P][N][T] (T = n_steps / tavg_steps).
 * Errors: TVBX_E_INVALID_ARG (dt <= 0, tavg_steps < 1, bad chunk_steps,
 * transient_samples >= T), TVBX_E_OOM, TVBX_E_CUDA. */
tvbx_status tvbx_run(tvbx_sweep* h, const tvbx_run_cfg* cfg, void* cuda_stream);

/* Continue the trajectory of h for n_steps more steps (Eq. 1-5 as in
 * tvbx_run) from the step where the last tvbx_run, tvbx_run_continue or
 * tvbx_restore left it, with the same dt, averaging, noise and seed. The
 * state, the delay ring buffers, the OU processes and the status bits carry
 * over, and the noise is keyed by the global step (counter-based Philox), so
 * tvbx_run of n1 steps followed by tvbx_run_continue of n2 steps follows the
 * same trajectory, bit for bit, as one tvbx_run of n1 + n2 steps. The series
 * [P][N][n_steps / tavg_steps] and the running sums behind the means, FC and
 * chi then cover the new samples only; transient_samples of them are left
 * out of the means. Asynchronous on cuda_stream like tvbx_run.
 * Errors: TVBX_E_BAD_STATE without a preceding run on h (a batch run does
 * not count) or when the steps so far are not a multiple of tavg_steps;
 * TVBX_E_INVALID_ARG for n_steps < 0, transient_samples out of range, or a
 * total of 2^32 - 1 steps or more; TVBX_E_OOM, TVBX_E_CUDA. */
tvbx_status tvbx_run_continue(tvbx_sweep* h, int64_t n_steps, int32_t transient_samples, void* cuda_stream);

/* Checkpoint / restore of a trajectory (no counterpart in the paper, whose
 * runs write observables only). A checkpoint is a host byte buffer holding
 * the state [14][N][P], the status words, the delay ring buffers, the OU
 * state, the step count and the run settings, tagged with a fingerprint of
 * the sweep's connectome, points and constants.
 *   tvbx_checkpoint_size: *bytes = the buffer size needed.
 *   tvbx_checkpoint: synchronises h's stream and copies into host_buf
 *     (caller-owned, at least that many bytes).
 *   tvbx_restore: loads a checkpoint into h, a sweep created with the same
 *     connectome, points and constants (any handle, e.g. in a new process);
 *     synchronous: it first waits for all work on the device, then fills h
 *     through the default stream. tvbx_run_continue on h then resumes bit
 *     for bit.
 * Errors: TVBX_E_BAD_STATE (checkpoint before any run), TVBX_E_INVALID_ARG
 * (NULL, short buffer, not a checkpoint, another sweep's checkpoint),
 * TVBX_E_OOM, TVBX_E_CUDA. */
tvbx_status tvbx_checkpoint_size(const tvbx_sweep* h, uint64_t* bytes);
tvbx_status tvbx_checkpoint(tvbx_sweep* h, void* host_buf, uint64_t bytes);
tvbx_status tvbx_restore(tvbx_sweep* h, const void* host_buf, uint64_t bytes);

/* Per-set summary of the last run, each output [n_sets] (any may be NULL):
 * mean E and I rates (Hz) over samples after the transient and regions,
 * the synchrony index chi = sqrt(Var_t(mean_k E_k) / mean_k Var_t(E_k)),
 * mean off-diagonal FC (Table 2 "mean_FC"), and the status bits.
 * chi and mean_fc need the FC pass: they are computed here if tvbx_fc has not
 * run since the last tvbx_run. Errors: TVBX_E_BAD_STATE before tvbx_run. */
tvbx_status tvbx_summary(tvbx_sweep* h, int32_t mem, float* mean_e_hz, float* mean_i_hz,
                         float* chi, float* mean_fc, uint32_t* status);

/* Copy a window of the E (pop 0) or I (pop 1) series, as tvbx_series_range;
 * the I series exists when the last run set keep_i_series (else
 * TVBX_E_BAD_STATE). */
tvbx_status tvbx_series_pop_range(const tvbx_sweep* h, int32_t pop, int64_t set_begin, int64_t set_count,
                                  int64_t t_begin, int64_t t_count, int32_t mem, float* out);

/* Copy the E series [n_sets][n_regions][n_samples] (kHz) of the last run. */
tvbx_status tvbx_series(const tvbx_sweep* h, int32_t mem, float* out);

/* Copy a window of the E series: sets [set_begin, set_begin + set_count) and
 * samples [t_begin, t_begin + t_count) into out [set_count][n_regions][t_count].
 * Errors: TVBX_E_INVALID_ARG when the window leaves the series. */
tvbx_status tvbx_series_range(const tvbx_sweep* h, int64_t set_begin, int64_t set_count,
                              int64_t t_begin, int64_t t_count, int32_t mem, float* out);

/* Copy the final state [n_sets][8][n_regions] of the last run, variables in
 * the order E, I, C_ee, C_ei, C_ii, W_e, W_i, OU (OU is the shared process of
 * each region when noise is shared). */
tvbx_status tvbx_state(const tvbx_sweep* h, int32_t mem, float* out);

/* Pearson FC (Eq. 6) of every set's E series after the transient:
 * fc_out [n_sets][n_regions][n_regions] (nullable), and, when
 * cfg->fcd_window > 0, FCD fcd_out [n_sets][n_windows][n_windows] with
 * n_windows = (T' - fcd_window) / fcd_step + 1 over T' = samples after the
 * transient (nullable). A region with zero variance has a zero FC row and
 * column and a unit diagonal, and sets TVBX_SET_ZERO_VAR.
 * Errors: TVBX_E_BAD_STATE before tvbx_run; TVBX_E_INVALID_ARG for a bad
 * window; TVBX_E_UNSUPPORTED for an unknown precision. */
tvbx_status tvbx_fc(tvbx_sweep* h, const tvbx_fc_cfg* cfg, int32_t mem, float* fc_out,
                    float* fcd_out, int32_t* n_windows);

/* Pearson FC (Eq. 6), FCD, synchrony index chi and mean off-diagonal FC of
 * series that are not the output of a sweep (the FC stage on its own).
 * series: DEVICE pointer, FP32, read-only, in cfg->series_layout:
 * [n_samples][n_regions][n_sets] (TVBX_LAYOUT_TNP, sets fastest) or the
 * set-blocked TVBX_LAYOUT_SET4. Outputs are DEVICE pointers owned by the caller, each nullable:
 * fc_out [n_sets][n_regions][n_regions], fcd_out [n_sets][W][W] with
 * W = (n_samples - fcd_window) / fcd_step + 1 (written to *n_windows when
 * non-NULL), chi and mean_fc [n_sets], set_status [n_sets] (OR-ed with
 * TVBX_SET_ZERO_VAR; not cleared). The shift of each row is the mean of up to
 * 64 evenly spaced samples. Scratch of n_sets x blocks x (n_regions^2 +
 * n_regions) floats (blocks = 1 without FCD, else ceil(n_samples /
 * fcd_step)) is allocated stream-ordered on cuda_stream (NULL = the legacy
 * default stream) from a memory pool the library owns per device, and freed
 * into it before return; the pool keeps that memory for later calls until the
 * process exits. The call synchronises cuda_stream before it returns.
 * Errors: TVBX_E_INVALID_ARG (NULL series, sizes < 1, bad window, a
 * tensor-core precision with n_regions > 112), TVBX_E_OOM, TVBX_E_CUDA,
 * TVBX_E_TIMEOUT (a bounded wait of the tensor-core kernel expired; the
 * outputs are then invalid), TVBX_E_UNSUPPORTED (unknown precision). */
tvbx_status tvbx_fc_series(const float* series, int32_t n_regions, int64_t n_sets, int64_t n_samples,
                           const tvbx_fc_cfg* cfg, float* fc_out, float* fcd_out, int32_t* n_windows,
                           float* chi, float* mean_fc, uint32_t* set_status, void* cuda_stream);

/* The transfer function of one population (Sec. "Transfer Function", Eq. 5
 * with Table 1) and its derivatives, evaluated on the GPU at n points, with
 * the same device code the integration uses. pop: 0 = excitatory (RS row,
 * W = W_e), 1 = inhibitory (FS row). Inputs x_e, x_i (total input rates,
 * kHz), W (pA), E_L (mV), each [n]; C [n][3] = (C_ee, C_ei, C_ii) (kHz^2,
 * nullable). out [n][8] = F, dF/dx_e, dF/dx_i, d2F/dx_e2, d2F/dx_e dx_i,
 * d2F/dx_i2, mu_V (mV), and sum_ij C_ij d2F/dx_i dx_j for Eq. 1 (0 when C is
 * NULL). F, the gradient, mu_V and the contracted term come from the code the
 * integrator runs (for tau_e == tau_i the reduced form of the template, else
 * the template itself, both with contracted second-order jets); the three
 * Hessian entries come from full second-order jets of the template.
 * All arrays live in memory of kind `mem`. model NULL = defaults. Synchronous. */
tvbx_status tvbx_transfer_function(const tvbx_model* model, int32_t pop, int64_t n, int32_t mem,
                                   const float* x_e, const float* x_i, const float* W,
                                   const float* E_L, const float* C, float* out);

/* Simulation kernel used by the last tvbx_run (TVBX_KERNEL_GENERAL or
 * TVBX_KERNEL_PREFETCH + v) and its tile size in sets. */
tvbx_status tvbx_last_kernel(const tvbx_sweep* h, int32_t* kernel, int32_t* sets_per_tile);

/* Number of kernels this library has launched in the process so far. */
uint64_t tvbx_launch_count(void);

/* Bytes this handle has copied host->device and device->host since it was
 * created (inputs uploaded by tvbx_run, outputs read to host memory). */
tvbx_status tvbx_transfer_bytes(const tvbx_sweep* h, uint64_t* h2d, uint64_t* d2h);

/* Kernel timing: when enabled, tvbx_run records a CUDA event pair around every
 * launch of the simulation kernel on the run's stream. tvbx_profile_read
 * synchronises that stream and returns the summed device time (ms), the
 * number of timed launches and the (set, region, step) updates they made,
 * accumulated since the last tvbx_profile_enable call. */
tvbx_status tvbx_profile_enable(tvbx_sweep* h, int32_t enable);
tvbx_status tvbx_profile_read(tvbx_sweep* h, double* sim_ms, int64_t* sim_launches,
                              double* region_steps);

/* FC without any device allocation. The paper has no counterpart: this is
 * a service of the library for callers that cannot allocate device memory
 * when they need an FC, e.g. hosts that fix their device-memory budget at
 * start-up and refuse later allocations (real-time or embedded services,
 * plugins under another framework's memory manager), or code where a
 * cudaMalloc would synchronise the device and stall other work.
 *   series   device, [n_samples][n_regions][n_sets] FP32 (sets fastest, the
 *            layout the engine keeps internally);
 *   fc_out   device, [n_sets][n_regions][n_regions] Pearson FC (Eq. 6) over
 *            all samples, with the conventions of tvbx_fc (zero-variance rows
 *            are zero, unit diagonal);
 *   chi, mean_fc  device, [n_sets] each, nullable (as in tvbx_summary).
 * Work is enqueued on cuda_stream (NULL = default stream); the call returns
 * without waiting. The only scratch, each set's moments, lives in a fixed
 * array of 8 Mi floats (32 MiB) reserved on every GPU that loads the library
 * until the process exits; a call needs n_sets * (n_regions^2 + n_regions)
 * floats of it, so n_sets <= 1,787 at 68 regions. Larger requests, more than
 * 90 regions, NULL buffers or non-positive sizes return TVBX_E_INVALID_ARG
 * with the limit in tvbx_last_error(). The moments are taken about the first
 * sample plus the mean deviation from it over up to 64 evenly spaced samples
 * (exactly the value of a constant row) and summed with compensation
 * (FP32 sums of 32-sample tiles, Kahan-added). The first call on each device
 * looks up the array's device address (cudaGetSymbolAddress with that device
 * current); make that first call before any stream capture. Later calls made
 * outside stream capture look the address up again, so a cudaDeviceReset
 * between calls is harmless; a call under capture uses the address of the
 * last call outside it, so do not reset the device between those. Every call
 * shares the array: calls that overlap on the GPU (other streams, other
 * threads) race and corrupt each other's results; serialise them. Each call
 * writes every scratch entry it reads, so nothing needs clearing between
 * calls. No cudaMalloc, cudaFree or allocating library routine is called. */
tvbx_status tvbx_fc_noalloc(const float* series, int32_t n_regions, int64_t n_sets, int64_t n_samples,
                            float* fc_out, float* chi, float* mean_fc, void* cuda_stream);

/* Release the handle and its device memory. NULL is accepted. */
tvbx_status tvbx_sweep_destroy(tvbx_sweep* h);

/* ---- Batches of sweeps ----------------------------------------------------
 * Runs several sweeps -- different connectomes (region counts), durations,
 * conduction speeds (delay horizons) and grids -- as one persistent kernel
 * launch captured in a CUDA graph (the batched form of the lock-step
 * integration of Eq. 1-5). Every (job, tile of sets) is a work item; CTAs
 * take items from a global counter, most expensive first, and integrate the
 * tile over the job's whole duration with the general kernel (state in
 * shared memory, any region count). The graph holds the per-job state, ring
 * and OU-table initialisation, the queue reset and the persistent kernel;
 * one tvbx_batch_run is one graph launch. Each job's results are read
 * through its own handle afterwards (tvbx_summary, tvbx_fc, tvbx_series ...),
 * and equal those of tvbx_run with kernel = TVBX_KERNEL_GENERAL bit for bit
 * (the tile width does not change any set's arithmetic). */
typedef struct tvbx_batch tvbx_batch;

/* jobs: n_jobs distinct sweep handles (borrowed: they must outlive the
 * batch); cfgs: their run configurations (copied; kernel and chunk_steps are
 * ignored, withhold_step must be 0, 1 <= n_steps < 2^31). Preparing a job
 * handle again with tvbx_run makes the next tvbx_batch_run rebuild the
 * graph. */
tvbx_status tvbx_batch_create(tvbx_sweep* const* jobs, const tvbx_run_cfg* cfgs, int32_t n_jobs,
                              tvbx_batch** out);

/* Autotuner: builds and times (two graph launches each, CUDA events) the
 * batch with each candidate tiling and keeps the fastest, rebuilding the full
 * batch with it. Candidates, in this order: six of the general body --
 * threads per CTA and shared-memory budget (256, 100 KB), (512, 100 KB),
 * (256, 200 KB), (512, 200 KB), (128, 64 KB), (256, 64 KB); the budget sets
 * each job's sets per CTA pb in {32, 16, 8} (the widest whose state fits) --
 * then two of the register-tile body (threads 512 and 768: each job with
 * N <= threads gets pb = 4 floor(threads / N) sets per CTA, 4 sets of one
 * region per thread; larger jobs keep the general body with a 200 KB budget).
 * Runs are shortened to trial_steps steps per job. threads_out, smem_kb_out:
 * the choice (smem_kb_out is the general body's budget); trial_ms [n_trials]
 * (host, nullable; 8 entries, INFINITY where a candidate does not fit).
 * Every candidate gives the same results bit for bit. */
tvbx_status tvbx_batch_tune(tvbx_batch* b, int64_t trial_steps, int32_t* threads_out, int32_t* smem_kb_out,
                            float* trial_ms, int32_t* n_trials);

/* Run every job (one graph launch; the first call builds the graph with
 * 512 threads and a 200 KB budget unless tvbx_batch_tune chose otherwise).
 * The jobs' later calls run on the batch's stream. Synchronises it. */
tvbx_status tvbx_batch_run(tvbx_batch* b);

/* Current tiling, work items, persistent grid size and graph nodes. */
tvbx_status tvbx_batch_info(const tvbx_batch* b, int32_t* threads, int32_t* smem_kb, int64_t* n_items,
                            int32_t* grid, int64_t* graph_nodes);

/* Release the batch (not its jobs; they keep their results and use the
 * default stream from then on). NULL is accepted. */
tvbx_status tvbx_batch_destroy(tvbx_batch* b);

/* Principal components of FC matrices (the FC coefficients the surrogate
 * predicts). fc: DEVICE [n_sets][n_regions][n_regions] Pearson FC (tvbx_fc
 * or tvbx_fc_series layout). The upper triangles (k < j, row by row; M =
 * n_regions (n_regions - 1) / 2 entries) are centred by their mean
 * (mean_out, DEVICE [M]); the n_comp leading eigenvectors of their
 * covariance matrix (comps_out, DEVICE [n_comp][M], orthonormal, largest
 * eigenvalue first, largest-magnitude entry positive) come from n_iter steps
 * of subspace iteration with n_comp + 12 vectors followed by a Rayleigh-Ritz
 * step; eigvals_out (HOST [n_comp], nullable) receives the eigenvalues of
 * the covariance (sum over sets / n_sets) and coef_out (DEVICE
 * [n_sets][n_comp], nullable) the coefficients of each set. Scratch of
 * n_sets * M + M * M floats is allocated on cuda_stream; the call
 * synchronises it. Errors: TVBX_E_INVALID_ARG (3 <= n_regions <= 512,
 * n_sets >= 2, 1 <= n_comp <= min(64, M), 1 <= n_iter <= 1000),
 * TVBX_E_NUMERIC (the FC vectors span fewer than n_comp + 12 directions),
 * TVBX_E_OOM, TVBX_E_CUDA. */
tvbx_status tvbx_fc_pca(const float* fc, int32_t n_regions, int64_t n_sets, int32_t n_comp, int32_t n_iter,
                        float* mean_out, float* comps_out, float* coef_out, float* eigvals_out,
                        void* cuda_stream);

/* Coefficients coef_out (DEVICE [n_sets][n_comp]) of further FC matrices fc
 * (DEVICE) on a basis from tvbx_fc_pca (mean, comps: DEVICE). */
tvbx_status tvbx_fc_pca_project(const float* fc, int32_t n_regions, int64_t n_sets, int32_t n_comp,
                                const float* mean, const float* comps, float* coef_out, void* cuda_stream);

/* ---- Fitness and grid search ----------------------------------------------
 * Sec. "Output": the simulated FC is compared with an externally obtained
 * reference FC and with the structural connectivity (FCSC) by the Pearson
 * coefficient (Eq. 6); Sec. "Validation using Functional Connectivity": the
 * fitness is that coefficient; Sec. "MPI": the results of a sweep are sorted
 * and the ten fittest reported (grid search).
 *
 * tvbx_fc_fitness: out[p][t] = Pearson coefficient between the strict upper
 * triangles (k < j) of fc[p] and of targets[t]: the fitness against a
 * reference FC, or the FCSC when the target is the connectome's weight
 * matrix. fc: DEVICE [n_sets][n_regions][n_regions] (e.g. tvbx_fc's output);
 * targets: DEVICE [n_targets][n_regions][n_regions], 1 <= n_targets <= 8,
 * 3 <= n_regions <= 1024; out: DEVICE [n_sets][n_targets], caller-owned.
 * A set whose triangle is constant or not finite gets NaN. A target whose
 * triangle is constant or not finite: TVBX_E_INVALID_ARG (checked before any
 * set is read; the call synchronises the stream once for this check).
 * Sums in FP32 over the centred triangle (the target's in FP64): the result
 * differs from the FP64 coefficient of the same FP32 inputs by about 1e-6.
 *
 * tvbx_top_k: the k largest finite entries of values (DEVICE [n],
 * 1 <= n < 2^31), largest first, ties to the lower index; 1 <= k <= 1024.
 * idx_out (DEVICE int64 [k]) and val_out (DEVICE [k]) are caller-owned;
 * positions beyond the number of finite entries get index -1 and NaN.
 * Selection compares values exactly (no rounding). Both calls are
 * asynchronous on cuda_stream (NULL = legacy default stream) apart from the
 * target check; scratch comes from the stream-ordered allocator. */
tvbx_status tvbx_fc_fitness(const float* fc, int64_t n_sets, int32_t n_regions, const float* targets,
                            int32_t n_targets, float* out, void* cuda_stream);
tvbx_status tvbx_top_k(const float* values, int64_t n, int32_t k, int64_t* idx_out, float* val_out,
                       void* cuda_stream);

/* ---- Table 2 analysis metrics ---------------------------------------------
 * Sec. "Analysis metrics", Table 2: mean_PLI (Sec. "Vast parameter space
 * exploration and analysis": the mean phase lag index), mean_UD_duration,
 * psd_fmax_ampmax and fit_psd_slope (log PSD = log(b / f^a)), computed on the
 * GPU from the excitatory rate series. The paper gives the metrics' names and
 * purpose only; this library's definitions:
 *  - samples: the last T' of each series, T' the largest number <=
 *    min(n_samples, 8192) whose prime factors are 2, 3 and 5; every discrete
 *    Fourier transform has length T' (the count is returned in *n_used);
 *  - PLI_kj = |mean_t sign(Im(z_k(t) conj(z_j(t))))| with z the analytic
 *    signal of the mean-removed series (one-sided spectrum doubled, inverse
 *    transform), sign(0) = 0; mean_PLI = mean over region pairs k < j;
 *  - PSD: per region the periodogram 2 dt |X(f)|^2 / T' of the mean-removed
 *    rate in Hz (dt the sample interval in s) at f_i = i / (T' dt),
 *    1 <= i < T'/2, averaged over regions; peak: the largest value for f in
 *    [1, 100] Hz (ties to the lower frequency); fit: least squares of
 *    log10 PSD = log10 b - a log10 f over the same band;
 *  - UP / DOWN: a region is UP while its rate exceeds its mean over the T'
 *    samples (the FP64 mean rounded to FP32); durations are lengths of
 *    maximal runs that neither start at the first nor end at the last
 *    sample, times dt; the set's means pool the runs of all regions.
 * Output row per set (TVBX_AN_COUNT floats, in this order); NaN where a
 * metric is undefined (no complete run, no band bin, N < 2 for the PLI). */
#define TVBX_AN_MEAN_PLI      0
#define TVBX_AN_PSD_FMAX      1  /* Hz */
#define TVBX_AN_PSD_AMPMAX    2  /* Hz^2 / Hz */
#define TVBX_AN_PSD_A         3  /* exponent a of b / f^a */
#define TVBX_AN_PSD_B         4  /* b, Hz^2 / Hz at 1 Hz */
#define TVBX_AN_UP_MS         5
#define TVBX_AN_DOWN_MS       6
#define TVBX_AN_N_UP          7  /* complete UP runs (exact integer) */
#define TVBX_AN_UP_SAMPLES    8  /* their total length in samples */
#define TVBX_AN_N_DOWN        9
#define TVBX_AN_DOWN_SAMPLES 10
#define TVBX_AN_COUNT        11

/* series: DEVICE or HOST [n_sets][n_regions][n_samples] FP32 rates in kHz
 * (the layout tvbx_series_range writes), sample interval dt_ms; out: DEVICE
 * [n_sets][TVBX_AN_COUNT], caller-owned; n_used: host, nullable. 1 <=
 * n_regions <= 752 (the phase-lag tiles of all regions must fit in shared
 * memory), n_samples >= 2. Sets are analysed in batches (the
 * analytic signals of up to 2 GiB of sets, whole waves of the phase-lag
 * kernel). A host series is uploaded batch by batch on a second stream into
 * two staging buffers, so the upload of one batch overlaps the analysis of
 * the previous one when the host memory is pinned (pageable memory works but
 * does not overlap); it must stay valid until cuda_stream has completed.
 * Asynchronous on cuda_stream (NULL = legacy default stream); scratch comes
 * from the stream-ordered allocator. */
tvbx_status tvbx_series_analysis(const float* series, int32_t n_regions, int64_t n_sets, int64_t n_samples,
                                 double dt_ms, float* out, int32_t* n_used, void* cuda_stream);

/* ---- BOLD signal and phFCD -------------------------------------------------
 * Sec. "Output": a Balloon-Windkessel kernel (Stephan et al. 2007) gives BOLD
 * series for comparison with fMRI, and the phase functional connectivity
 * dynamics (phFCD) of those series is computed for comparison.
 *
 * tvbx_bold: forward Euler of the Balloon-Windkessel model (Friston et al.
 * 2000; Stephan et al. 2007), time in seconds, drive z = the E rate in kHz:
 *   ds/dt = z - kappa s - gamma (f - 1),  df/dt = s,
 *   tau dv/dt = f - v^(1/alpha),
 *   tau dq/dt = f E(f)/E0 - v^(1/alpha) q / v,  E(f) = 1 - (1 - E0)^(1/f),
 *   y = V0 (k1 (1 - q) + k2 (1 - q/v) + k3 (1 - v)),
 *   k1 = 4.3 theta0 E0 TE, k2 = eps r0 E0 TE, k3 = 1 - eps;
 * one step per rate sample (dt_ms), one BOLD value after every `decim`
 * steps. series: DEVICE [n_samples][n_regions][n_sets] (sets fastest, as
 * TVBX_LAYOUT_TNP, e.g. a stretch of rates the caller keeps); bold_out: DEVICE
 * [n_samples / decim][n_regions][n_sets]; state: DEVICE [4][n_regions]
 * [n_sets] = (s, f - 1, v - 1, q - 1), nullable; with reset_state = 1 (or no
 * state) the integration starts at rest, otherwise from *state, and the final
 * state is written back, so long runs can be fed in pieces. params NULL =
 * tvbx_bold_defaults (kappa 0.65 /s, gamma 0.41 /s, tau 0.98 s, alpha 0.32,
 * E0 0.34, V0 0.02, theta0 40.3 /s, r0 25 /s, TE 0.04 s, eps 1).
 *
 * tvbx_phfcd: for each set, the last T'' samples of each region's BOLD
 * series (T'' the largest number <= min(n_tr, 8192) whose prime factors are
 * 2, 3 and 5), mean removed; the band-limited analytic signal (DFT bins
 * 0 < i < T''/2 with i / (T'' tr_s) in [f_lo_hz, f_hi_hz] doubled, all
 * others 0, inverse DFT); `discard` samples dropped at each end, T' =
 * T'' - 2 discard kept (returned in *n_used, host, nullable); phases theta
 * (0 where the signal is 0); dFC_kj(t) = cos(theta_k - theta_j); output
 * out[p][e] = cosine similarity of the upper triangles (k < j) of dFC(t1)
 * and dFC(t2) for every t1 < t2, e = t1 T' - t1 (t1 + 1) / 2 + t2 - t1 - 1.
 * bold: DEVICE [n_tr][n_regions][n_sets]; out: DEVICE [n_sets][T'(T'-1)/2].
 * 2 <= n_regions <= 200 (two 64-sample phase tiles of all regions must fit
 * in shared memory).
 * Both calls are asynchronous on cuda_stream (NULL = legacy default stream). */
typedef struct {
    double kappa, gamma, tau, alpha, E0, V0, theta0, r0, TE, eps;
} tvbx_bold_params;
tvbx_status tvbx_bold_defaults(tvbx_bold_params* out);
tvbx_status tvbx_bold(const float* series, int32_t n_regions, int64_t n_sets, int64_t n_samples, double dt_ms,
                      int32_t decim, const tvbx_bold_params* params, float* state, int32_t reset_state,
                      float* bold_out, void* cuda_stream);
tvbx_status tvbx_phfcd(const float* bold, int32_t n_regions, int64_t n_sets, int64_t n_tr, double tr_s,
                       double f_lo_hz, double f_hi_hz, int32_t discard, float* out, int32_t* n_used,
                       void* cuda_stream);

/* ---- Refit of the transfer-function polynomial ------------------------------
 * Sec. "Transfer Function": the template's effective threshold is the
 * second-order polynomial of Table 1 in the normalised mu_V, sigma_V,
 * tau_V^N, fitted to simulations of single AdEx neurons (Zerlaut et al.
 * 2018). These calls redo that fit on the GPU.
 *
 * tvbx_cell_rates: output rates (kHz, host rate_khz_out [n_points]) of
 * n_cells independent cells at each point (input rates nu_e_khz, nu_i_khz per
 * input synapse, constant current -W_pA; host arrays [n_points]). Each cell
 * is an adaptive exponential integrate-and-fire neuron
 *   C dV/dt = g_L (E_L - V) + g_L Delta exp((V - V_T) / Delta)
 *             + g_e (E_e - V) + g_i (E_i - V) - W,
 * spike at V >= V_T + 5 Delta (reset to V_reset, refractory t_ref), with
 * exponential conductances (time constants tau_e, tau_i) that jump by Q_e,
 * Q_i per input spike; forward Euler with step dt_ms; per step the input
 * counts are Poisson with means K_e nu_e dt and K_i nu_i dt, drawn from words
 * 0 and 1 of Philox4x32-10 (counter (step, cell index, 0, 0), key = seed,
 * cell index = point n_cells + c) by comparison with the integer thresholds
 * floor(P(N <= k) 2^32), k < 32. Spikes after transient_ms count. Runs on
 * the legacy default stream and returns when the rates are on the host.
 * tvbx_cell_defaults: regular-spiking (pop 0) or fast-spiking (pop 1) cell
 * (C 200 pF, g_L 10 nS, E_L -64 mV, V_T -50 mV, Delta 2 or 0.5 mV, V_reset
 * -65 mV, t_ref 5 ms, Q_e 1.5 nS, Q_i 5 nS, tau_e = tau_i = 5 ms, E_e 0,
 * E_i -80 mV, K_e 400, K_i 100).
 *
 * tvbx_tf_fit: host computation (no device use). For each point with a rate F
 * in (0, 1 / (2 tau_V)): the template's mu_V, sigma_V, tau_V, tau_V^N (FP64,
 * model m, leak E_L[p], current W_pA[p]) and the effective threshold
 * mu_V + sqrt(2) sigma_V erfcinv(2 tau_V F); P_out[10] = least-squares
 * coefficients (mV, Table 1 column order) of the threshold polynomial;
 * *n_used = points used (nullable). Fewer than 10 usable points:
 * TVBX_E_NUMERIC. */
typedef struct {
    double C, gL, EL, VT, Delta, Vreset, t_ref, Qe, Qi, tau_e, tau_i, Ee, Ei, Ke, Ki;
} tvbx_cell_params;
tvbx_status tvbx_cell_defaults(int32_t pop, tvbx_cell_params* out);
tvbx_status tvbx_cell_rates(const tvbx_cell_params* cell, int64_t n_points, const double* nu_e_khz,
                            const double* nu_i_khz, const double* W_pA, int32_t n_cells, double T_ms,
                            double transient_ms, double dt_ms, uint64_t seed, double* rate_khz_out);
tvbx_status tvbx_tf_fit(const tvbx_model* m, int64_t n_points, const double* nu_e_khz, const double* nu_i_khz,
                        const double* W_pA, const double* E_L, const double* rate_khz, double P_out[10],
                        int32_t* n_used);

/* tvbx_tf_refit: host computation (no device use), the fit's second stage
 * (Sec. "Transfer Function": the polynomial is fitted to single-cell rates;
 * Zerlaut's procedure refines the threshold fit on the rates themselves).
 * Starting from P_init[10] (e.g. tvbx_tf_fit's result), the coefficients
 * that minimise sum_p (F_p(P) - rate_p)^2, F_p(P) the template's rate
 * erfc((V_thre(P) - mu_V) / (sqrt(2) sigma_V)) / (2 tau_V), over every point
 * with a finite rate >= 0 (silent and saturated points included), by
 * Levenberg-Marquardt with the analytic Jacobian, at most max_iter steps
 * (0: P_out = P_init, i.e. the rate error of given coefficients).
 * P_out[10] (mV, Table 1 column order); *rms_out = root-mean-square rate
 * error (kHz) at P_out and *n_used = points used (both nullable). Fewer than
 * 10 usable points or non-finite rates at P_init: TVBX_E_NUMERIC. */
tvbx_status tvbx_tf_refit(const tvbx_model* m, int64_t n_points, const double* nu_e_khz, const double* nu_i_khz,
                          const double* W_pA, const double* E_L, const double* rate_khz, const double P_init[10],
                          int32_t max_iter, double P_out[10], double* rms_out, int32_t* n_used);

/* ---- Surrogate network ---------------------------------------------------
 * The paper has no surrogate model; it motivates guided exploration of the
 * parameter space (Sec. "Discussion"). This is the learned form of the
 * exploration: an ensemble of multilayer perceptrons, trained on the GPU by
 * the library's own kernels, that maps sweep parameters (e.g. g, b_e,
 * tau_w_e, E_L_i, v) to summary statistics of a simulation (e.g. mean rates,
 * chi, mean FC, FC principal-component coefficients) and proposes where the
 * sweep should be refined; every proposal is then simulated and checked.
 *
 * Network: inputs mapped to [-1, 1] by the domain box; n_layers hidden layers
 * of n_hidden units, a = max(0, a_prev W^T + b); linear output layer that
 * predicts the outputs standardised by a training set's per-output
 * mean and population standard deviation (see tvbx_surrogate_train). Loss: mean squared error over rows
 * and outputs. Optimiser: AdamW (decoupled weight decay on weight matrices
 * only; beta1 0.9, beta2 0.999, eps 1e-8). Weights: FP32 master copy and a
 * BF16 copy read by the matrix products; FP32 accumulation. Initial weights:
 * He-uniform from Philox (key = seed), zero biases. Members differ by their
 * initial weights and shuffles.
 * Flattened parameter layout of one member (host arrays below): layer by
 * layer, W [out][in] row-major, then b [out]. Handles are not thread-safe;
 * each owns a CUDA stream and every call returns after its work completed. */
typedef struct tvbx_surrogate tvbx_surrogate;
typedef struct {
    int32_t n_in;        /* inputs, 1..64 */
    int32_t n_hidden;    /* units per hidden layer, 1..1024 */
    int32_t n_layers;    /* hidden layers, 1..8 */
    int32_t n_out;       /* outputs, 1..256 */
    int32_t n_members;   /* ensemble size, 1..16 */
    uint64_t seed;       /* initial weights, shuffles, candidates */
    const double* in_lo; /* [n_in] domain box (copied); finite, in_lo < in_hi */
    const double* in_hi; /* [n_in] */
} tvbx_surrogate_cfg;

/* Create; *out receives the handle. Errors: TVBX_E_INVALID_ARG (sizes, box),
 * TVBX_E_OOM, TVBX_E_CUDA. */
tvbx_status tvbx_surrogate_create(const tvbx_surrogate_cfg* cfg, tvbx_surrogate** out);

/* Parameters per member and ensemble size (either pointer nullable). */
tvbx_status tvbx_surrogate_info(const tvbx_surrogate* s, int64_t* n_params, int32_t* n_members);

/* Flags of tvbx_surrogate_train. */
#define TVBX_TRAIN_SHUFFLE 1       /* each member visits the rows in its own
                                      pseudo-random order per pass (else in order) */
#define TVBX_TRAIN_KEEP_SCALE 2    /* keep the output standardisation of the
                                      earlier training call (fine-tuning on a
                                      few new rows must not move the scale the
                                      network was trained in); ignored on a
                                      handle that was never trained */

/* Train every member on X [n][n_in], Y [n][n_out] (FP32; mem = TVBX_MEM_HOST
 * or TVBX_MEM_DEVICE): recompute the output standardisation from Y (unless
 * flags has TVBX_TRAIN_KEEP_SCALE), then `epochs` passes in mini-batches of
 * `batch` rows (the last one may be shorter), one AdamW step (learning rate
 * lr, weight decay weight_decay) per mini-batch; flags: TVBX_TRAIN_* bits.
 * loss_out (host, nullable) receives the mean training loss of each pass
 * [epochs] (over members and mini-batches, in standardised units). */
tvbx_status tvbx_surrogate_train(tvbx_surrogate* s, int32_t mem, const float* X, const float* Y, int64_t n,
                                 int32_t epochs, int32_t batch, float lr, float weight_decay, int32_t flags,
                                 float* loss_out);

/* Ensemble mean y_mean [n][n_out] and variance y_var [n][n_out] (nullable)
 * across members of the predictions in output units, for X [n][n_in]; all on
 * the host or all on the device (mem). */
tvbx_status tvbx_surrogate_predict(tvbx_surrogate* s, int32_t mem, const float* X, int64_t n, float* y_mean,
                                   float* y_var);

/* Propose n_propose points where output `output` is closest to `threshold`
 * and the ensemble disagrees most: n_candidates points drawn uniformly in the
 * candidate box (Philox, counter = (candidate, round, input), key = seed) --
 * cand_lo/cand_hi (host [n_in], both or neither; cand_lo[i] == cand_hi[i]
 * fixes input i, e.g. to map a 2-D slice), else the domain box -- are scored
 * by -|mean - threshold| / sd + var_weight sqrt(var) / sd (sd = the output's
 * training standard deviation) and the best n_propose (ties to the lower
 * candidate index) are written, best first, to points_out [n_propose][n_in]
 * (host) with their scores (host, nullable). */
tvbx_status tvbx_surrogate_propose(tvbx_surrogate* s, int64_t n_candidates, uint64_t round, int32_t output,
                                   float threshold, float var_weight, const double* cand_lo,
                                   const double* cand_hi, int32_t n_propose, float* points_out,
                                   float* scores_out);

/* Rank caller-given candidates X [n][n_in] (host) by the proposal score of
 * tvbx_surrogate_propose (-|mean - threshold| / sd + var_weight sqrt(var) / sd
 * for output `output`) and write the indices of the best n_propose (best
 * first; ties to the lower index) to idx_out [n_propose] (host) with their
 * scores (host, nullable). exclude (host uint8 [n], nullable): candidates
 * with a non-zero byte are never chosen, e.g. points of a map that the
 * simulator has already judged. A candidate whose prediction is not finite
 * scores -inf and ranks last. Errors: TVBX_E_INVALID_ARG when n < 1, n >
 * 2^26, or n_propose exceeds the candidates not excluded. */
tvbx_status tvbx_surrogate_rank(tvbx_surrogate* s, const float* X, int64_t n, const uint8_t* exclude, int32_t output,
                                float threshold, float var_weight, int32_t n_propose, int64_t* idx_out,
                                float* scores_out);

/* Read (get_out) and/or replace (set_in) the FP32 parameters of one member
 * (host arrays of tvbx_surrogate_info's n_params; either nullable). Setting
 * also rounds the BF16 copy and clears that member's optimiser state. */
tvbx_status tvbx_surrogate_params(tvbx_surrogate* s, int32_t member, float* get_out, const float* set_in);

/* Loss and gradient (host, [n_params], flattened layout) of one member on
 * host X [n][n_in], Y [n][n_out] with the current standardisation, without
 * an update; n <= 2^20. */
tvbx_status tvbx_surrogate_gradients(tvbx_surrogate* s, int32_t member, const float* X, const float* Y, int64_t n,
                                     float* loss, float* grads);

/* Release the handle. NULL is accepted. */
tvbx_status tvbx_surrogate_destroy(tvbx_surrogate* s);

#ifdef __cplusplus
}
#endif
#endif /* TVBX_H */

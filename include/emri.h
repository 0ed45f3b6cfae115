/*
 * emri.h -- C-ABI of libemri, the GB300-native (sm_103a) batched
 * Analytic-Kludge (AK) EMRI log-likelihood of Saltas & Oliveri,
 * "emri_mc: A GPU-based Python code for Bayesian inference of EMRI
 * waveforms" (arXiv:2311.17174).
 *
 * One likelihood evaluation follows the paper's pipeline (Sec. 3,
 * "Overview" and "Waveform computation"): integrate the AK orbit of Eq. (1),
 * form the detector-projected harmonic sum of Eq. (2) with the LISA response
 * and Doppler phase, propagate with the damping Xi of Eqs. (4)-(6) and the
 * GW-speed delay, Fourier transform, and take the noise-weighted inner
 * product of Eq. (8) against the data.  Every step runs in the library's own
 * CUDA kernels; there is no CPU fallback and no cuFFT/cuBLAS.
 *
 * Conventions (all entry points):
 *  - Every call returns an int status (enum emri_status); on failure
 *    emri_last_error() gives a message (thread-local, valid until the next
 *    call on the same thread).
 *  - The caller owns every pointer it passes: device pointers for batch
 *    inputs and outputs (for example torch tensors), host pointers where a
 *    parameter says "host".  The library owns contexts, datasets, workspaces
 *    and plans and frees them in the matching destroy call.
 *  - Calls that take a stream (cudaStream_t passed as void*, NULL = the
 *    legacy default stream) are asynchronous on it; results are ready once
 *    the stream has been synchronised.
 *  - Walker parameters are structure-of-arrays, theta[EMRI_NPARAM][W]
 *    (row p holds parameter p of every walker, W contiguous doubles), in the
 *    order of enum emri_param.  Angles in radians, masses in solar masses,
 *    frequencies in Hz.
 *  - Without a usable CUDA device every call fails with EMRI_ECUDA.
 */
#ifndef EMRI_H
#define EMRI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define EMRI_NPARAM 16

/* Parameter rows of theta (paper Sec. 2: theta = {M, mu, S, ...}; the first
 * three are the ones the orbit needs, Sec. 3 "Extending the parameters"). */
enum emri_param {
  EMRI_P_M = 0,      /* central mass M [M_sun], detector frame          */
  EMRI_P_MU = 1,     /* orbiting mass mu [M_sun]                         */
  EMRI_P_SPIN = 2,   /* S/M^2 in [0, 1]                                  */
  EMRI_P_E0 = 3,     /* eccentricity at t0 (at the LSO in backward mode) */
  EMRI_P_NU0 = 4,    /* orbital frequency nu at t0 [Hz] (forward mode)   */
  EMRI_P_PHI0 = 5,   /* orbital phase Phi at t0 (backward: at the LSO)   */
  EMRI_P_GAMMA0 = 6, /* periastron angle gamma~ at t0 (backward: LSO)    */
  EMRI_P_ALPHA0 = 7, /* Lense-Thirring angle alpha at t0 (backward: LSO) */
  EMRI_P_THETA_S = 8, EMRI_P_PHI_S = 9,   /* source direction (ecliptic) */
  EMRI_P_THETA_K = 10, EMRI_P_PHI_K = 11, /* spin direction              */
  EMRI_P_LAMBDA = 12,/* angle between L and S                            */
  EMRI_P_Z = 13,     /* redshift                                          */
  EMRI_P_XI0 = 14,   /* damping parameter Xi_0 of Eq. (6)                */
  EMRI_P_ALPHA_T = 15/* GW-speed parameter alpha_T (constant) of Eq. (5) */
};

enum emri_status {
  EMRI_OK = 0,
  EMRI_EINVAL = 1,     /* bad argument (size, pointer, option)            */
  EMRI_ENOMEM = 2,     /* device or host allocation failed               */
  EMRI_EBUDGET = 3,    /* request exceeds the context's HBM budget       */
  EMRI_EAGAIN = 4,     /* serving queue full, retry                       */
  EMRI_ETIMEDOUT = 5,  /* poll timeout                                     */
  EMRI_ECUDA = 6,      /* CUDA error or no device                         */
  EMRI_ENOTFOUND = 7   /* unknown ticket / not started                    */
};

enum emri_precision {
  EMRI_FP64 = 0,  /* every step in FP64                                    */
  EMRI_MIXED = 1  /* orbit and phases FP64/fixed point, harmonic sum and
                     FFT FP32, inner products accumulated in FP64           */
};

enum emri_mode {
  EMRI_FORWARD = 0,          /* integrate forward from (nu0, e0) at t0     */
  EMRI_BACKWARD_FROM_LSO = 1 /* initial conditions at the LSO (paper
                                Sec. 3): the last sample t0 + (n-1) dt has
                                e = e0 and nu = nu_LSO(e0), and Phi0,
                                gamma~0, alpha0 are the angles there; nu0 is
                                ignored; the orbit is integrated backwards,
                                so no plunge occurs in the window          */
};

/* per-walker status bits */
#define EMRI_ST_PLUNGE 1u   /* orbit reached the LSO inside the window; the
                               waveform is zero from that sample on        */
#define EMRI_ST_BADPARAM 2u /* parameters outside their domain; outputs 0
                               (lnL = -inf is not used: lnL = 0, check bit) */
#define EMRI_ST_NONFINITE 4u/* the orbit became non-finite                 */

typedef struct emri_ctx emri_ctx;
typedef struct emri_dataset emri_dataset;

/* Uniform time grid: samples t_j = t0 + j dt, j = 0..n-1 (paper Sec. 3: the
 * orbit is an initial-value problem evaluated on a time grid). */
typedef struct {
  int64_t n;   /* samples per channel, a power of two in [2^10, 2^22]      */
  double dt;   /* sampling step [s]                                        */
  double t0;   /* time of sample 0 [s]; sets the LISA orbital phase        */
} emri_grid;

typedef struct {
  int precision;    /* enum emri_precision                                   */
  int n_max;        /* harmonic cutoff n_max of Eq. (2), 1..32               */
  int doppler;      /* 1: Doppler phase modulation on, 0: off               */
  int pn_terms;     /* 1: full AK equations; 0: Newtonian radiation reaction */
  int mode;         /* enum emri_mode                                         */
  int knot_spacing; /* samples per orbit knot interval (power of two, 64..
                       1024); 0 = library default for the precision         */
  double n_xi;      /* exponent n of Eq. (6); default 2                      */
  double omega_m;   /* flat Lambda-CDM matter density; default 0.315         */
  double h0;        /* Hubble constant [km/s/Mpc]; default 67.4              */
} emri_opts;

/* Fill *o with the defaults: FP64, n_max 10, Doppler on, full AK, forward,
 * default knot spacing, n_xi 2, Omega_m 0.315, H0 67.4. */
void emri_opts_default(emri_opts* o);

/* Thread-local message of the last failed call on this thread ("" if none). */
const char* emri_last_error(void);

/* Library version string. */
const char* emri_version(void);

/* Create a context on CUDA device `device`.  hbm_budget_bytes caps the
 * device memory the library holds for workspaces and resident datasets
 * (0 = 80% of the device's free memory at creation).  Builds the FFT twiddle
 * and quadrature tables.  *out receives the context (caller destroys).
 * Debug aid: with the environment variable EMRI_DEBUG_POISON set to a
 * non-zero value at creation, the context's shared workspace is filled with
 * 0xFF bytes (NaN as FP32/FP64) before every call, so that a kernel reading
 * intermediate data that the same call did not write yields NaN instead of a
 * stale value from an earlier call; it costs one memset per call. */
int emri_ctx_create(int device, size_t hbm_budget_bytes, emri_ctx** out);

/* Stop serving if running (requests still queued fail with
 * EMRI_ENOTFOUND), free every workspace, table and the context.  Datasets are
 * owned by the caller: destroy them first (a dataset must not outlive its
 * context).  NULL is a no-op. */
int emri_ctx_destroy(emri_ctx* ctx);

/* Overlap of the likelihood's steps across walker groups (a scheduling
 * choice with no counterpart in the paper, whose Sec. 3 evaluates the
 * walkers' likelihoods independently).  The walkers of each wave of a call
 * are split into `groups` groups of consecutive walkers.  The first group's
 * orbits (step S1) run first, then every other walker's in one launch, on a
 * context-owned stream; each group's waveform (S2-S4) runs on the caller's
 * stream once its orbits are done, and its FFT passes and reduction (S5-S7)
 * on a second context-owned stream once its waveform is written.  Both
 * context streams have the device's highest priority, so a group's passes
 * are dispatched ahead of the next group's waveform.  groups = 1 runs every
 * step in order on the caller's stream.  Applies to emri_loglike_batch(_fd)
 * and the stretch-step entry points of this precision (EMRI_FP64 or
 * EMRI_MIXED), except on a stream that is being captured (those calls use
 * 1).  Each walker is computed by the same kernels on the same data, so the
 * results are bitwise the same for every `groups`.  Before the call returns,
 * the caller's stream is made to wait for both context streams, so
 * stream-ordered use of the outputs is safe as usual.  The context streams
 * and 132 events are created at the first call that uses them (no device
 * memory).  groups: 1..64, or 0 = by the call's size: 2 groups when each
 * holds at least 2^30 samples (walkers of a wave x n), else 1; smaller
 * groups lose more to the extra orbit launch and the stream hand-offs than
 * the overlap gains.  Default 1 (FP64: every kernel is bound by the FP64
 * pipe) and 0 (mixed).  EMRI_EINVAL otherwise. */
int emri_ctx_set_pipeline(emri_ctx* ctx, int precision, int groups);

/* Number of CUDA kernels the library has launched on this context so far
 * (host counter, incremented at each launch). */
int emri_ctx_launches(const emri_ctx* ctx, int64_t* count);

/* Device bytes the context holds (workspaces, tables, datasets) and its
 * budget; either output may be NULL. */
int emri_ctx_memory(const emri_ctx* ctx, size_t* used, size_t* budget);

/* Kernel kinds of the likelihood path, for per-kernel timing. */
enum emri_kernel {
  EMRI_K_PROLOGUE = 0,   /* S0 per-walker constants                      */
  EMRI_K_DELAY = 1,      /* S0 per-walker delay table                    */
  EMRI_K_ORBIT = 2,      /* S1 orbit integration                         */
  EMRI_K_WAVE = 3,       /* S2-S4 harmonic sum and response              */
  EMRI_K_FFT1 = 4,       /* S5 FFT pass 1                                */
  EMRI_K_FFT2_IP = 5,    /* S5-S6 FFT pass 2 fused with inner products   */
  EMRI_K_FINALIZE = 6,   /* S7 reduction and lnL                         */
  EMRI_K_FFT2_STORE = 7, /* S5 FFT pass 2 to natural order (emri_fft_batch) */
  EMRI_NKERNEL = 8
};

/* Enable (1) or disable (0) per-kernel timing on this context and reset the
 * accumulators.  While enabled, every launch of the likelihood path is
 * bracketed by CUDA events recorded on the stream it is launched on.  Under
 * the pipelined schedule (emri_ctx_set_pipeline) kernels of different walker
 * groups run at the same time, so a launch's interval also covers the
 * kernels beside it; set groups to 1 for a per-kernel breakdown. */
int emri_ctx_profile(emri_ctx* ctx, int enable);

/* Wait for the recorded events and return, per enum emri_kernel, the summed
 * device time [ms] and the launch count since profiling was enabled (host
 * arrays of EMRI_NKERNEL entries; either may be NULL). */
int emri_ctx_kernel_times(emri_ctx* ctx, double* ms, int64_t* launches);

/* Resident dataset (paper Sec. 3: the waveform of the fiducial parameters is
 * the mock data the sampler compares against; the PSD weights Eq. (8)).
 *   data:  data_kind 0: packed spectrum D_k = DFT(d_I + i d_II) in natural
 *          order, n complex doubles (interleaved re, im);
 *          data_kind 1: time series, two channels d[2][n] doubles.
 *          Host or device pointer; copied.
 *   psd:   one-sided noise PSD S_n(f_k) at f_k = k/(n dt), k = 0..n/2
 *          (n/2+1 doubles, host or device); copied.
 *   fmin, fmax: band [Hz]; bins with fmin <= |f_k| <= fmax, excluding DC
 *          and Nyquist, get the weight w_k = 2 dt^2 df / S_n(|f_k|), others
 *          zero, so that sum_k w_k Re(conj(A_k) B_k) over all n bins is the
 *          one-sided 4 Re sum a~* b~ / S_n df of the two channels.
 * The dataset lives in device memory counted against the HBM budget. */
int emri_dataset_create(emri_ctx* ctx, const emri_grid* grid, const void* data, int data_kind,
                        const double* psd, double fmin, double fmax, emri_dataset** out);
/* Free a dataset (waits for the device); NULL is a no-op.  Call it before
 * destroying the dataset's context. */
int emri_dataset_destroy(emri_dataset* ds);

/* <d|d> of the dataset (host double). */
int emri_dataset_dd(const emri_dataset* ds, double* dd_out);

/* Per-walker propagation constants (step S0; Eqs. (4)-(6)) into
 * out_dev[6][W] (device): d_L [cm], Xi, d_GW = Xi d_L [cm],
 * dt_GW = -(alpha_T/2) t_lookback(z) [s], r_hi, r_lo with
 * r = frac(dt_GW / (n dt)) split into two doubles. */
int emri_prologue(emri_ctx* ctx, const emri_grid* grid, const double* theta_dev, int w,
                  const emri_opts* opts, double* out_dev, void* stream);

/* Time-domain waveform of W walkers (steps S1-S4; Eqs. (1)-(2)): the two
 * LISA channels at unit distance (1 cm), packed as z_j = h_I(t_j) + i
 * h_II(t_j), into z_out_dev[W][n] complex: double2 (16 B) for EMRI_FP64,
 * float2 (8 B) for EMRI_MIXED.  status_dev (nullable) receives W status
 * words.  W = 0 is a no-op. */
int emri_ak_waveform(emri_ctx* ctx, const emri_grid* grid, const double* theta_dev, int w,
                     const emri_opts* opts, void* z_out_dev, uint32_t* status_dev, void* stream);

/* In-place batched FFT (step S5) of `batch` contiguous complex sequences of
 * length n (power of two, 2^10..2^22): Z_k = sum_j z_j exp(s 2 pi i j k / n)
 * with s = -1 for direction -1 (forward) and +1 for direction +1
 * (unnormalised inverse).  precision EMRI_FP64: double2, EMRI_MIXED: float2.
 * Natural order in and out. */
int emri_fft_batch(emri_ctx* ctx, void* z_dev, int64_t n, int batch, int precision, int direction,
                   void* stream);

/* ----------------------------------------------------- allocation-free FFT
 * The paper has no counterpart to this entry point; it serves callers that
 * cannot call cudaMalloc -- a plugin limited to the memory its host
 * application hands it, a process whose device memory is fully reserved by
 * another allocator, or a real-time loop that must never enter the
 * allocator.  Same transform, layout and arguments as emri_fft_batch, but no
 * context: the scratch the second pass writes (32 MiB: at least one whole
 * sequence, several when they are shorter) and the twiddle tables are
 * file-scope static device arrays of the library
 * (EMRI_NOALLOC_SCRATCH_BYTES of scratch plus 216 KiB of tables, held on
 * every GPU that loads the library until the process exits).  Nothing is
 * allocated by the call.
 *  - Limit: one sequence must fit the scratch, n * 16 B (FP64) or n * 8 B
 *    (EMRI_MIXED) <= EMRI_NOALLOC_SCRATCH_BYTES, i.e. n <= 2^21 in FP64 and
 *    n <= 2^22 in FP32; larger n returns EMRI_EINVAL with a message.  Any
 *    batch size is accepted (processed in chunks that fit the scratch).
 *  - The first call on a device (the current device) resolves the arrays'
 *    addresses with cudaGetSymbolAddress and fills the tables, synchronising
 *    `stream`; make that first call before any stream capture (a first call
 *    on a capturing stream returns EMRI_EINVAL and does nothing).
 *  - All calls on a device share the scratch: calls whose work overlaps on
 *    the GPU (different streams, unordered host threads) race. */
#define EMRI_NOALLOC_SCRATCH_BYTES (32u << 20)
int emri_fft_batch_noalloc(void* z_dev, int64_t n, int batch, int precision, int direction, void* stream);

/* Batched log-likelihood (steps S0-S7; Eq. (8)) of W walkers against a
 * dataset:  lnL = <d|h> - <h|h>/2 (the constant -<d|d>/2 left out) with
 * h = h_u / d_GW delayed by dt_GW,
 *   <d|h_u> = sum_k w_k Re(conj(D_k) H_u,k exp(-2 pi i k_s r)),
 *   <h_u|h_u> = sum_k w_k |H_u,k|^2,
 * H_u = DFT of the unit-distance packed channels, k_s the signed bin index.
 * Outputs (device, W doubles each): lnl_dev; dh_dev, hh_dev (nullable) the
 * unit-distance sums <d|h_u>, <h_u|h_u>; status_dev (nullable).  Reduction
 * order is fixed per (n, opts), so a walker's result does not depend on the
 * other walkers in the call.  W = 0 is a no-op. */
int emri_loglike_batch(emri_ctx* ctx, const emri_dataset* ds, const double* theta_dev, int w,
                       const emri_opts* opts, double* lnl_dev, double* dh_dev, double* hh_dev,
                       uint32_t* status_dev, void* stream);

/* ------------------------------------- frequency-dependent propagation
 * Paper Sec. 2 allows alpha_M and alpha_T to depend on the GW frequency
 * (alpha_M = F(z, f), alpha_T = G(z, f), e.g. a power series in f/f_*),
 * acting on the waveform in frequency space.  Model (coefficients constant
 * in z, per walker):
 *   alpha_M(f) = sum_{m=1..q_m} a_m (f/f_*)^m: every bin is scaled by
 *                (1+z)^(-alpha_M(|f|)/2) (the z-independent case of the
 *                damping integral; the constant part stays Xi of Eq. (6));
 *   alpha_T(f) = alpha_T + sum_{m=1..q_t} b_m (f/f_*)^m: the GW-speed delay
 *                becomes dt_GW(f) = -(alpha_T(|f|)/2) t_LB(z), i.e. the bin
 *                factor exp(-2 pi i f dt_GW(f)) at the signed f_k.
 * emri_loglike_batch_fd is emri_loglike_batch with these factors applied per
 * bin inside the fused FFT pass (<h|h> includes the amplitude factor); the
 * phase, up to ~1e18 cycles, is evaluated exactly mod 1 in 128-bit fixed
 * point.  coef_dev (device, [q_m + q_t][W], caller-owned): a_1..a_qm then
 * b_1..b_qt per walker.  q_m = q_t = 0 reproduces emri_loglike_batch.
 * Errors: EMRI_EINVAL for q outside [0, 3], f_star <= 0, NULL coefficients. */
typedef struct {
  int q_m;                 /* alpha_M terms, 0..3                           */
  int q_t;                 /* extra alpha_T terms, 0..3                     */
  double f_star;           /* pivot frequency f_* [Hz], > 0                  */
  const double* coef_dev;  /* [q_m + q_t][W] device doubles                 */
} emri_fdprop;

int emri_loglike_batch_fd(emri_ctx* ctx, const emri_dataset* ds, const double* theta_dev, int w,
                          const emri_opts* opts, const emri_fdprop* fd, double* lnl_dev, double* dh_dev,
                          double* hh_dev, uint32_t* status_dev, void* stream);

/* ------------------------------------------------------- uneven batching
 * Several independent chains, each with its own dataset (its own n), walker
 * count and options, evaluated by one launch of a captured CUDA graph with
 * one branch per chain, so that the chains' kernels overlap on the device.
 * The graph is captured on the first call with a given item list (pointers,
 * counts and options) and replayed while the list stays the same; the values
 * behind the pointers may change between calls.  Each chain has its own
 * workspace (its time series bounded to ~512 MiB per wave).  Knot spacing and
 * wave size follow the autotuner's plan for the chain's shape when one
 * exists.  Pointers in emri_work are device pointers owned by the caller;
 * outputs and determinism as emri_loglike_batch: each chain's results equal
 * those of the chain evaluated alone. */
typedef struct {
  const emri_dataset* ds;
  const double* theta_dev; /* [EMRI_NPARAM][w] */
  int w;
  emri_opts opts;
  double* lnl_dev;
  double* dh_dev;          /* nullable */
  double* hh_dev;          /* nullable */
  uint32_t* status_dev;    /* nullable */
  const emri_fdprop* fd;   /* nullable (host struct): the chain's frequency-dependent
                              propagation, as in emri_loglike_batch_fd; its
                              coef_dev [q_m + q_t][w] is part of the graph's key */
} emri_work;

int emri_loglike_multi(emri_ctx* ctx, const emri_work* items, int n_items, void* stream);

/* ------------------------------------------------------- ensemble step
 * One step of the affine-invariant ensemble sampler the paper uses for its
 * posterior (Sec. 3, "Posterior sampling": emcee's stretch move, Goodman &
 * Weare 2010, Commun. Appl. Math. Comput. Sci. 5, 65), on the device:
 *   the W walkers form two halves S0 = [0, h), S1 = [h, W), h = W/2; S0 is
 *   updated against the current S1, then S1 against the updated S0.  Walker
 *   k of the active half takes the partner j = floor(u[0][k] * |other|) of
 *   the other half and z = ((a - 1) u[1][k] + 1)^2 / a (density ~ z^-1/2 on
 *   [1/a, a]); the proposal Y = X_j + z (X_k - X_j) in the free parameters
 *   (others copied from X_k) is accepted iff
 *   (d - 1) ln z + lnP(Y) - lnP(X_k) - ln u[2][k] > 0, d = number of free
 *   parameters.  lnP = lnL of emri_loglike_batch plus a flat prior on the
 *   box lo <= theta_p <= hi for the free p; a proposal outside the box, or
 *   with status ST_BADPARAM / ST_NONFINITE, is rejected.
 * theta_dev [EMRI_NPARAM][W] and lnp_dev [W] (device, caller-owned) hold the
 * ensemble and its lnP on entry and are updated in place (lnp_dev of the
 * starting ensemble comes from emri_loglike_batch).  u_dev [3][W] (device):
 * uniforms in [0, 1) drawn by the caller, one triple per walker and step.
 * accepted_dev [W] (nullable): 1 where the walker moved.  The proposal is
 * formed with correctly rounded operations in the order written above.
 * Errors: EMRI_EINVAL for W = 1, a <= 1, an empty free mask, bits above
 * parameter 15, or an empty prior box; W = 0 is a no-op.  Asynchronous on
 * `stream`; uses the context's workspace (sized for the larger half). */
typedef struct {
  double a;                 /* stretch scale, > 1 (2 is the usual choice)    */
  uint32_t free_mask;       /* bit p set: parameter p (theta order) moves    */
  double lo[EMRI_NPARAM];   /* flat prior box of the free parameters         */
  double hi[EMRI_NPARAM];
} emri_stretch_cfg;

int emri_stretch_step(emri_ctx* ctx, const emri_dataset* ds, double* theta_dev, double* lnp_dev, int w,
                      const emri_opts* opts, const emri_stretch_cfg* cfg, const double* u_dev,
                      int32_t* accepted_dev, void* stream);

/* One block of one half-step of emri_stretch_step, for an ensemble whose
 * walkers are spread over several GPUs (paper Sec. 3, "Posterior sampling":
 * the walkers of the parallel stretch move are independent within a half,
 * so each GPU can move its own block of each half).  Updates walkers
 * k0 <= k < k1 of half `half` (0: [0, W/2), 1: [W/2, W); the block must lie
 * inside it) against the whole other half, exactly as emri_stretch_step does
 * for them: theta_dev[EMRI_NPARAM][W] and lnp_dev[W] hold the whole ensemble
 * (the other half must be current on this device), and only the block's
 * columns, lnp and accepted entries are written; u_dev[3][W] as for
 * emri_stretch_step; fd (nullable) as in emri_stretch_step_fd.  Running
 * half 0 over blocks that cover it, making the
 * updated half 0 current everywhere, then half 1 likewise, gives the same
 * ensemble bit for bit as one emri_stretch_step.  Errors as
 * emri_stretch_step, plus EMRI_EINVAL for a block outside the half; an empty
 * block is a no-op. */
int emri_stretch_half(emri_ctx* ctx, const emri_dataset* ds, double* theta_dev, double* lnp_dev, int w, int half,
                      int k0, int k1, const emri_opts* opts, const emri_stretch_cfg* cfg, const emri_fdprop* fd,
                      const double* u_dev, int32_t* accepted_dev, void* stream);

/* emri_stretch_step with the frequency-dependent propagation of
 * emri_loglike_batch_fd (paper Sec. 2, alpha_M(f), alpha_T(f)) held fixed per
 * walker: fd->coef_dev [q_m + q_t][W] (device, caller-owned), and the
 * proposal of walker k is evaluated with walker k's coefficients (the
 * coefficients are not moved).  emri_stretch_half takes the same model
 * through its nullable fd argument. */
int emri_stretch_step_fd(emri_ctx* ctx, const emri_dataset* ds, double* theta_dev, double* lnp_dev, int w,
                         const emri_opts* opts, const emri_stretch_cfg* cfg, const emri_fdprop* fd,
                         const double* u_dev, int32_t* accepted_dev, void* stream);

/* ------------------------------------------------------------- serving
 * A continuous-batching request loop on the context's device (the serving
 * configuration of paper Sec. 3's likelihood evaluations for many chains):
 * requests arriving while others run are admitted as slots and HBM free up,
 * and run concurrently on the device.  emri_serve_start allocates one device
 * pool of the serving budget and charges it to the context until stop; each
 * admitted request holds a contiguous range of it (its parameters, results
 * and workspace) while it runs, so an admitted request never fails for
 * memory and the loop never allocates device memory.  Requests are admitted
 * in arrival order, except that later requests that fit may pass one that
 * does not fit yet, at most 32 times, after which admission waits for it. */
typedef struct {
  int slots;            /* concurrent requests on the device (streams), >= 1  */
  int queue_capacity;   /* pending requests before submit returns EAGAIN      */
  size_t budget_bytes;  /* pool bytes, at most the context's remaining budget;
                           0 = half of the context's remaining budget         */
} emri_serve_cfg;

typedef struct {
  int64_t arrival_ns;   /* submit time (CLOCK_MONOTONIC)                      */
  int64_t start_ns;     /* admission (work enqueued on the device)            */
  int64_t done_ns;      /* results observed complete                          */
  int32_t status;       /* emri_status of the request                         */
  int32_t slot;         /* stream slot that ran it                            */
} emri_req_stats;

int emri_serve_start(emri_ctx* ctx, const emri_serve_cfg* cfg);
int emri_serve_stop(emri_ctx* ctx);

/* Enqueue W walkers (theta_host[EMRI_NPARAM][W], host, copied before return)
 * against a dataset.  *ticket identifies the request.  EMRI_EAGAIN when the
 * queue is full; EMRI_EBUDGET when the request alone exceeds the budget. */
int emri_serve_submit(emri_ctx* ctx, const emri_dataset* ds, const double* theta_host, int w,
                      const emri_opts* opts, uint64_t* ticket);

/* emri_serve_submit with the frequency-dependent propagation of
 * emri_loglike_batch_fd (paper Sec. 2, alpha_M(f), alpha_T(f)): q_m, q_t in
 * [0, 3], f_star > 0, coef_host[q_m + q_t][W] (host, copied before return;
 * NULL allowed when q_m + q_t = 0).  Results equal emri_loglike_batch_fd on
 * the same walkers. */
int emri_serve_submit_fd(emri_ctx* ctx, const emri_dataset* ds, const double* theta_host, int w,
                         const emri_opts* opts, int q_m, int q_t, double f_star, const double* coef_host,
                         uint64_t* ticket);

/* Pool bytes a request of W walkers against `ds` with `opts` holds while it
 * runs (host query; a request larger than the pool is refused at submit). */
int emri_serve_request_bytes(emri_ctx* ctx, const emri_dataset* ds, int w, const emri_opts* opts,
                             size_t* bytes);

/* Wait up to timeout_us (<0: forever) for a request; on completion copy its
 * W log-likelihoods to lnl_host, statuses to status_host (nullable) and the
 * timestamps to stats (nullable), then release the ticket.
 * EMRI_ETIMEDOUT if not done in time, EMRI_ENOTFOUND for an unknown ticket. */
int emri_serve_poll(emri_ctx* ctx, uint64_t ticket, double* lnl_host, uint32_t* status_host,
                    emri_req_stats* stats, int64_t timeout_us);

/* ----------------------------------------------------------- autotuner
 * Time the library's schedule choices (knot spacing, walkers per wave, FFT
 * split) for this grid, n_max and precision on the context's device and keep
 * the fastest as the context's plan for that shape; with cache_path
 * non-NULL the plans are also read from / appended to that JSON-lines file.
 * A call whose (n, n_max, precision) has no plan uses the plan tuned for the
 * same n and precision at the nearest n_max, if any.
 * choice_out (nullable, host) receives {knot_spacing, wave_walkers, fft_n1}. */
int emri_autotune(emri_ctx* ctx, const emri_grid* grid, int n_max, int precision,
                  const char* cache_path, int64_t* choice_out);

#ifdef __cplusplus
}
#endif
#endif /* EMRI_H */

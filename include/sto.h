/*
 * sto.h - C ABI of libsto, a B300 (sm_103a) simulator of N coupled
 * spin-torque oscillators (STOs) used as a physical reservoir, after
 * T. G. de Jong et al., "Virtual reservoir acceleration for CPU and GPU:
 * case study for coupled spin-torque oscillator reservoir", arXiv 2312.01121.
 *
 * The method (Sec. 3.1, Eq. (gov)): every oscillator k carries a unit
 * magnetisation m_k = (m^x, m^y, m^z) that follows the Landau-Lifshitz-Gilbert
 * equation with spin-transfer torque
 *     dm_k/dt = -gamma' m_k x b_k - alpha gamma' m_k x (m_k x b_k),
 *     gamma'  = gamma / (1 + alpha^2),
 *     b_k     = [H_appl + (H_K - 4 pi M) m_k^z] e_z              (Eq. gov)
 *             + A_cp sum_i W[k,i] m_i^x e_x                      (Eq. coup)
 *             + g A_in sum_j w_in[k,j] u_j e_x                   (Eq. in)
 *             + H_s(m_k) p x m_k,
 *     H_s(m)  = hbar eta I / (2 e (1 + lambda m.p) M V)           (Eq. gov).
 * Eq. (coup) is printed with m_k^x inside the sum; the library reads it as
 * m_i^x, the matrix-vector product W m^x that Sec. 3.3 describes.  Time
 * stepping is classic RK4 with a fixed step dt (Sec. 3.2).  The input u is
 * a discrete series (Sec. 3.1): sample t is held for `substeps` RK4 steps,
 * after which the reservoir state (one component of every m_k, Sec. 3.1:
 * "N-states are used as the nodes") is recorded.
 *
 * Units: fields in Oe, time in s, gamma in rad/(Oe s), M in emu/cm^3,
 * V in cm^3, I in A, hbar in J s, e in C; H_s carries the factor 1e7 (J to
 * erg) so that it comes out in Oe (134.87 Oe at the Table values).
 *
 * Precision: W and the coupling matrix-vector product are FP32 (FP32
 * products, FP32 accumulation); the per-oscillator torque, the RK4 stage
 * combination and the state are FP64 (double-float on the FP32 pipes,
 * about 48 significand bits, FP64 in memory).  Sampled states are returned
 * in FP32.  sto_create_f64 selects an FP64 coupling instead (the precision
 * of the paper's own benchmark, Sec. 3.3).
 *
 * Conventions for every entry point:
 *   - Return value: STO_OK (0) or a negative STO_E* code; sto_strerror()
 *     describes it.  No call throws or aborts the process.  There is no CPU
 *     fallback: without a usable CUDA device every compute call fails with
 *     STO_ECUDA.
 *   - Pointers marked "host or device" may point to host memory (pageable or
 *     pinned) or to device memory of the handle's device; the library
 *     inspects them with cudaPointerGetAttributes.  Arrays are dense,
 *     row-major, float32 unless stated otherwise.
 *   - Arrays passed to sto_create are copied; the caller keeps ownership of
 *     every pointer it passes and may free it once the call has returned.
 *   - All device work is ordered on the stream given at creation.  Calls
 *     that produce a status synchronise that stream before returning.
 *   - A handle is not thread-safe: one host thread at a time per handle.
 *   - After STO_ETIMEOUT or STO_ECUDA the handle's state is unspecified;
 *     sto_set_state() makes it usable again.
 */
#ifndef STO_H_
#define STO_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define STO_ABI_VERSION 4

#if defined(__GNUC__)
#define STO_API __attribute__((visibility("default")))
#else
#define STO_API
#endif

/* Status codes. */
#define STO_OK 0
#define STO_EINVAL (-1)      /* invalid argument (null pointer, size, range) */
#define STO_ENOMEM (-2)      /* device or host allocation failed */
#define STO_ECUDA (-3)       /* a CUDA runtime call failed (see sto_strerror) */
#define STO_ETIMEOUT (-4)    /* a device-side wait exceeded its time limit */
#define STO_ENONFINITE (-5)  /* NaN or Inf found in an input */
#define STO_ENOTSUP (-6)     /* size or option outside what the library supports */
#define STO_ETOOBIG (-7)     /* N above the static scratch of sto_run_noalloc */
#define STO_ESINGULAR (-8)   /* the ridge system of the readout is not positive definite */

/* Model parameters.  Defaults (sto_default_params) are Table "Summary of
 * parameters" of Sec. 3.1 and the step of Sec. 3.2; substeps, n_in,
 * input_gain and sample_component are not fixed by the paper. */
typedef struct sto_params {
  double gamma;       /* gyromagnetic ratio, rad/(Oe s)          1.764e7 */
  double alpha;       /* Gilbert damping                          0.005 */
  double Ms;          /* saturation magnetisation M, emu/cm^3     1448.3 */
  double Hk;          /* anisotropy field H_K, Oe                 18616 */
  double Happl;       /* applied field, Oe                        200 */
  double eta;         /* spin polarisation                        0.537 */
  double lambda;      /* spin-transfer torque asymmetry           0.288 */
  double current;     /* I, A                                     2.5e-3 */
  double volume;      /* V, cm^3                     pi*60^2*2 nm^3 */
  double e_charge;    /* elementary charge, C             1.60217733e-19 */
  double hbar;        /* reduced Planck constant, J s     1.05457266e-34 */
  double p[3];        /* pinned-layer direction     (1, 0, 6.123234e-17) */
  double A_cp;        /* coupling amplitude, Oe                   1 */
  double A_in;        /* input amplitude, Oe                      1 */
  double input_gain;  /* g, multiplies A_in                       1 */
  double dt;          /* RK4 step, s                              1e-11 */
  int32_t substeps;   /* RK4 steps per input sample (S)           100 */
  int32_t n_in;       /* input channels N_in                      1 */
  int32_t sample_component; /* recorded component: 0=x, 1=y, 2=z   0 */
  int32_t reserved;   /* must be 0 */
} sto_params;

/* Launch-plan overrides for sto_create_ex.  Zero fields mean "choose". */
typedef struct sto_config {
  int32_t grid;        /* CTAs of the persistent kernel (1 .. #SMs, <= N) */
  int32_t timeout_ms;  /* limit of every device-side wait (default 2000) */
  int32_t l2_keep_mb;  /* W larger than L2: MB of W kept L2-resident across
                          stages (0 = default, 110 MB; -1 = none) */
  int32_t tmem_w;      /* FP32 W larger than L2: 0 (default) keeps a few
                          panels of each CTA's rows of W in the SM's tensor
                          memory for the whole call (up to 128 columns per
                          consumer warp: 6 panels of 68 x 128 at N = 10^4,
                          from the middle of the streamed ones), so they are
                          not streamed again; -1 streams every panel.  The
                          results are the same bits. */
  int32_t reserved[4]; /* must be 0 */
} sto_config;

/* The launch plan chosen for a handle (read-only, for tuning and reports). */
typedef struct sto_info {
  int64_t N;
  int32_t grid;          /* CTAs, one per SM, co-resident */
  int32_t rows_max;      /* most oscillators owned by one CTA */
  int32_t panel_cols;    /* columns of W per streamed panel (128, or 64
                            for sto_create_f64) */
  int32_t panels;        /* panels per row block (ceil(N / panel_cols)) */
  int32_t ring_slots;    /* shared-memory panel buffers per CTA */
  int32_t resident;      /* 1: each CTA keeps its rows of W on chip */
  int32_t smem_bytes;    /* dynamic shared memory per CTA */
  int32_t sm_count;      /* SMs of the device */
  int64_t w_bytes;       /* bytes of W streamed per RK4 stage (4 N^2, or
                            8 N^2 for sto_create_f64) */
  int32_t xbuf_timed;    /* placements of the exchange buffer timed at the
                            handle's first sto_run or sto_adjoint (8 when W
                            is on chip and G > 1: the stage time depends on
                            where the polled lines fall in the L2; 0 before
                            that or otherwise) */
  int32_t xbuf_slot;     /* the placement kept (the fastest) */
  int32_t tmem_panels;   /* panels of each CTA's rows of W held in tensor
                            memory for the whole call (sto_config.tmem_w);
                            0 when W is on chip, L2-resident or not FP32 */
} sto_info;

typedef struct sto_handle sto_handle; /* opaque */

/* Fill *out with the defaults above.  Never fails. */
STO_API void sto_default_params(sto_params* out);

/* Create a simulator for one reservoir of N oscillators (Sec. 3.1).
 *   N       >= 1.  The largest N is set by shared memory: about 21000 with
 *           148 CTAs on a B300 (STO_ENOTSUP beyond).
 *   params  model parameters; checked for finiteness and ranges.
 *   W       N x N coupling matrix, row k = target oscillator, column i =
 *           source (Eq. coup), host or device.  The paper's W has a zero
 *           diagonal; any finite matrix is accepted.
 *   w_in    N x n_in input weights (Eq. in), host or device.
 *   m0      initial state, 3 x N (all m^x, then m^y, then m^z), host or
 *           device; NULL selects Eq. (initial): every m_k =
 *           (sin phi0 cos phi0, sin phi0 sin phi0, cos phi0), phi0 = 2pi/360.
 *   stream  cudaStream_t to order all work on (NULL = legacy default).
 *   out     receives the handle; *out is NULL on failure.
 * Errors: STO_EINVAL, STO_ENONFINITE (NaN/Inf in W, w_in or m0),
 *         STO_ENOMEM, STO_ENOTSUP, STO_ECUDA. */
STO_API int sto_create(int64_t N, const sto_params* params, const float* W,
               const float* w_in, const float* m0, void* stream,
               sto_handle** out);

/* sto_create with launch-plan overrides (cfg may be NULL). */
STO_API int sto_create_ex(int64_t N, const sto_params* params, const float* W,
                  const float* w_in, const float* m0, void* stream,
                  const sto_config* cfg, sto_handle** out);

/* Coupling products of sto_create_f64. */
#define STO_PRODUCT_DF 1   /* W kept as an exact pair of floats (hi + lo, the
                              FP64 value to 48 significand bits); products and
                              row sums in double-float on the FP32 pipes */
#define STO_PRODUCT_F64 2  /* W kept in FP64; FP64 fused multiply-adds */

/* A reservoir with an FP64 coupling matrix: the paper's benchmark runs the
 * whole method in FP64 (Sec. 3.3, Table 1: RK4 with dt = 1e-11 s, u = 0,
 * random W with zero diagonal scaled to spectral radius 1), and this replica
 * keeps W, the stage values exchanged between CTAs and the coupling sums
 * at FP64 width instead of FP32.  8 N^2 bytes of W are read per RK4 stage.
 *   N, params, w_in, stream, cfg, out   as for sto_create_ex (w_in and the
 *               input series u of sto_run stay float32; both are exact in
 *               FP64).
 *   W           N x N row-major float64, host or device; copied.
 *   m0          3 x N float64 initial state, host or device, or NULL for
 *               Eq. (initial).
 *   product     STO_PRODUCT_DF or STO_PRODUCT_F64 (see above).  The B300's
 *               FP64 pipe is far slower than its FP32 pipes, so the
 *               double-float product is the fast one; STO_PRODUCT_F64 gives
 *               IEEE FP64 products and sums.
 * sto_run, sto_run_group, sto_set_state[_f64], sto_get_state[_f64],
 * sto_set_params, sto_get_info and sto_destroy work on the handle as on any
 * other.  Largest N about 18000 with 148 CTAs (STO_ENOTSUP beyond).
 * Errors: as sto_create_ex; STO_EINVAL for an unknown product;
 *         sto_adjoint and sto_set_tableau on the handle return STO_ENOTSUP. */
STO_API int sto_create_f64(int64_t N, const sto_params* params, const double* W,
                           const float* w_in, const double* m0, void* stream,
                           const sto_config* cfg, int32_t product, sto_handle** out);

/* Replace the model parameters (not N, n_in or the plan).  Lets a caller
 * sweep I, A_cp, the gain, dt, substeps ... without re-uploading W.
 * n_in must equal the value given at creation.  Errors: STO_EINVAL. */
STO_API int sto_set_params(sto_handle* h, const sto_params* params);

/* Set / read the state, 3 x N float32 (m^x block, m^y block, m^z block),
 * host or device.  The internal state is FP64; sto_get_state rounds it. */
STO_API int sto_set_state(sto_handle* h, const float* m);
STO_API int sto_get_state(const sto_handle* h, float* m);
/* Exact FP64 state, 3 x N doubles, host or device (checkpoint / resume). */
STO_API int sto_set_state_f64(sto_handle* h, const double* m);
STO_API int sto_get_state_f64(const sto_handle* h, double* m);

/* Advance the reservoir over T input samples (Sec. 3.1, Sec. 3.2).
 *   u           T x n_in float32 input series, host or device (may be NULL
 *               only if T == 0).
 *   T           >= 0; T == 0 returns STO_OK and does nothing.
 *   states_out  T x N float32, host or device, or NULL: after sample t,
 *               states_out[t*N + k] = component `sample_component` of m_k.
 * For every sample t: the input field of Eq. (in) is formed from u[t] and
 * held for `substeps` classic RK4 steps of size dt, each stage evaluating
 * the full coupling field A_cp W m^x of Eq. (coup).  The state advances in
 * place.  The whole call is one persistent kernel launch; it synchronises
 * the stream once at the end to read the device error word.
 * Errors: STO_EINVAL, STO_ETIMEOUT, STO_ECUDA, STO_ENOMEM (host buffers
 *         larger than any earlier call need a device staging buffer). */
STO_API int sto_run(sto_handle* h, const float* u, int64_t T, float* states_out);

/* Gradients returned by sto_adjoint. */
typedef struct sto_grads {
  double dA_cp;      /* dL/dA_cp */
  double dcurrent;   /* dL/dI (per ampere) */
  double* dw_in;     /* N x n_in output, host or device, or NULL */
  double* dm0;       /* 3 x N output (dL/dm at the start), host or device, or NULL */
} sto_grads;

/* Gradients for parameter search (Sec. 1 and Sec. 2 call the exploration of
 * the parameter space the time-consuming part): the exact derivatives of
 *     L = sum_{t,k} dL_dstates[t*N + k] * states_out[t*N + k]
 * for the run sto_run(h, u, T, states_out) would do from the current state,
 * with respect to A_cp, the current I, the input weights w_in and the
 * initial state.  This is the discrete adjoint of the RK4 stepper (not an
 * adjoint ODE), so it matches finite differences of sto_run to rounding.
 * With dL_dstates = dLoss/dstates of a readout loss evaluated at the fitted
 * readout weights, the result is the gradient of the refitted loss
 * (envelope theorem).
 *   u, T          as for sto_run (T >= 1).
 *   dL_dstates    T x N float32, host or device.
 *   ckpt_every    K >= 1: the state is checkpointed every K input samples;
 *                 each K-sample segment is recomputed once with its
 *                 trajectory recorded (K * substeps * N * 40 bytes of device
 *                 memory), then swept backwards.  Cost: two forward runs
 *                 (the checkpoint pass, then the recomputation with
 *                 recording) and one reverse run with a W^T product per
 *                 stage.  With W on chip and several segments, each
 *                 segment's recomputation runs on a second stream beside
 *                 the reverse pass of the segment after it (another
 *                 recording buffer of the same size; the same results).
 *   out           receives dA_cp and dcurrent; dw_in / dm0 are written if
 *                 non-NULL.
 * The state ends where sto_run would leave it.  The first call builds a
 * tiled copy of W^T (another 4 N^2 bytes).
 * Errors: STO_EINVAL, STO_ENOMEM, STO_ETIMEOUT, STO_ECUDA, STO_ENOTSUP. */
STO_API int sto_adjoint(sto_handle* h, const float* u, int64_t T, const float* dL_dstates,
                        int32_t ckpt_every, sto_grads* out);

/* Advance n independent reservoirs (each its own handle: its own W, N,
 * parameters and launch plan) over the same input series u (T x n_in, host
 * or device; every handle must have the same n_in and device).  The n
 * persistent launches are captured into one CUDA graph and run back to
 * back; states_out[i] (T x N_i, host or device, or NULL; states_out itself may
 * be NULL) receives reservoir i's states.  The uneven-N, own-W half of a
 * parameter sweep.
 * Errors: STO_EINVAL (duplicate handles, mismatched n_in), STO_ENOMEM,
 *         STO_ETIMEOUT, STO_ECUDA, STO_ENOTSUP. */
STO_API int sto_run_group(sto_handle* const* hs, int32_t n, const float* u, int64_t T,
                          float* const* states_out);

/* ------------------------------------------------------------------------
 * A group of reservoirs with their own W (the uneven-N, own-W half of a
 * parameter sweep; Sec. 1 and Sec. 2: exploring the parameter space is the
 * time-consuming part) advanced by ONE persistent cooperative launch per
 * call.  The grid is cut into `lanes` lanes of SMs/lanes CTAs; each lane runs
 * its reservoirs one after another, each on all of the lane's CTAs, so
 * reservoirs on different lanes run at the same time (small reservoirs,
 * which are latency-bound alone, share the GPU instead of holding all of
 * it).  Reservoirs are assigned to lanes longest first onto the least
 * loaded lane.  Results equal sto_run's on a handle with the same launch
 * plan (grid = the lane width) bit for bit.
 * ------------------------------------------------------------------------ */
typedef struct sto_group sto_group; /* opaque */

/* Make a group of n distinct handles (same device, same n_in, FP32
 * coupling).  lanes = 0 picks the largest lane count up to min(n, 8) for
 * which every reservoir has at least one oscillator per CTA and at most 120
 * per CTA.  Each handle is re-planned for the lane width with W in shared
 * memory (its W re-tiled on the device; sto_run on it keeps working, with
 * that plan, and gives the group's bits; a different plan can change the
 * coupling sums' last bits).  The
 * group keeps the handle pointers: destroy the group before its handles.
 * Errors: STO_EINVAL (null, duplicate handles, mismatched n_in or device),
 *         STO_ENOTSUP (an FP64 handle, or no lane count fits), STO_ENOMEM,
 *         STO_ECUDA. */
STO_API int sto_group_create(sto_handle* const* hs, int32_t n, int32_t lanes, sto_group** out);

/* Advance every member over the same T input samples u (T x n_in, host or
 * device); states_out[i] (T x N_i, host or device, or NULL; states_out
 * itself may be NULL) receives member i's samples.  One cooperative launch;
 * the call synchronises the first member's stream once at the start (to
 * reuse its argument records) and once at the end.
 * Errors: STO_EINVAL, STO_ENOTSUP (a member re-planned or given a tableau
 *         since creation), STO_ENOMEM, STO_ETIMEOUT, STO_ECUDA. */
STO_API int sto_group_run(sto_group* g, const float* u, int64_t T, float* const* states_out);

/* sto_group_create for a group that shares the GPU with a sweep in one
 * launch (sto_run_sweep_group): its lanes occupy ctas CTAs (0 = one per SM,
 * as sto_group_create), the other SMs are left to the sweep.  lanes = 0
 * picks the lane count as sto_group_create does for that many CTAs.
 * Errors: as sto_group_create; STO_EINVAL for ctas outside 0 .. #SMs. */
STO_API int sto_group_create_ex(sto_handle* const* hs, int32_t n, int32_t lanes, int32_t ctas, sto_group** out);

/* The lane count, the CTAs per lane, and (lane_of, n entries, or NULL) the
 * lane each member runs on.  Errors: STO_EINVAL. */
STO_API int sto_group_get_info(const sto_group* g, int32_t* lanes, int32_t* lane_width, int32_t* lane_of);

/* Release the group (not its handles; NULL is allowed). */
STO_API void sto_group_destroy(sto_group* g);

/* Use an explicit Runge-Kutta method other than classic RK4 (Sec. 3.2 uses
 * classic RK4; the paper's conclusion notes that the approach applies to
 * any reservoir evolved by an explicit method).  stages = s in 1..4;
 * a: s x s row-major Butcher matrix, strictly lower triangular (entries on
 * or above the diagonal must be 0); b: s weights.  stages = 0 (a, b NULL)
 * restores classic RK4.  Each RK step then takes s exchange stages.  The
 * adjoint (sto_adjoint) is available for classic RK4 only (STO_ENOTSUP).
 * Errors: STO_EINVAL (implicit or non-finite tableau, s out of range). */
STO_API int sto_set_tableau(sto_handle* h, int32_t stages, const double* a, const double* b);

/* Replace the input weights w_in (N x n_in float32, host or device).
 * Errors: STO_EINVAL, STO_ENONFINITE, STO_ECUDA. */
STO_API int sto_set_input_weights(sto_handle* h, const float* w_in);

/* ------------------------------------------------------------------------
 * Batched parameter sweep (Sec. 1 and Sec. 2: exploring the parameter space
 * is the time-consuming part).  R reservoirs share one coupling matrix W and
 * the input weights, and differ in their current I_r and input gain g_r; all
 * are driven by the same input series.  Per RK4 stage the coupling of all
 * reservoirs is one dense product W [m^x_0 ... m^x_{R-1}] on the tensor cores
 * (tcgen05, BF16 W, the stage values split into two BF16 terms, FP32
 * accumulation), followed by the double-float torque and RK4 combination of
 * every (reservoir, oscillator) pair.  W is rounded to BF16 once, at
 * creation: results match the single-reservoir method run with that W.
 * ------------------------------------------------------------------------ */
typedef struct sto_batch sto_batch; /* opaque */

/* Create a sweep of R reservoirs of N oscillators.
 *   params      shared parameters (substeps, dt, A_cp, n_in, ...).
 *   current     R currents I_r in A, or NULL for params->current.
 *   input_gain  R gains g_r, or NULL for params->input_gain.
 *   W           N x N float32 (host or device), rounded to BF16.
 *   w_in        N x n_in float32 (host or device), shared.
 *   m0          R x 3 x N float32 initial states (reservoir-major; host or
 *               device) or NULL for Eq. (initial).
 * Limits: N <= 32768, R <= 65536 and R N <= 2^29 (STO_ENOTSUP otherwise).
 * Errors: STO_EINVAL, STO_ENONFINITE, STO_ENOMEM, STO_ENOTSUP, STO_ECUDA. */
STO_API int sto_batch_create(int64_t N, int32_t R, const sto_params* params,
                             const double* current, const double* input_gain,
                             const float* W, const float* w_in, const float* m0,
                             void* stream, sto_batch** out);

/* Advance every reservoir over T input samples of the shared series u
 * (T x n_in, host or device).  states_out: T x R x N float32 (sample,
 * reservoir, oscillator; host or device) or NULL.  The call is one
 * persistent cooperative launch (captured with its barrier reset as a CUDA
 * graph): per RK4 stage every CTA multiplies its tiles of D = W X on the
 * tensor cores and finishes them (torque, RK4 combination, next X), then
 * all CTAs meet at a grid barrier.  The first call without a plan runs the
 * autotuner (sto_batch_set_plan(b, 0, 0)).  4 * substeps * T <= 2^30.
 * Errors: STO_EINVAL, STO_ENOMEM, STO_ENOTSUP, STO_ETIMEOUT, STO_ECUDA. */
STO_API int sto_run_batched(sto_batch* b, const float* u, int64_t T, float* states_out);

/* A whole parameter sweep (Sec. 1 and Sec. 2: exploring the parameter
 * space is the time-consuming part) in ONE persistent cooperative launch,
 * captured as a CUDA graph: the shared-W reservoirs of b on the SMs that the
 * own-W group g leaves free (#SMs - its lanes x lane width CTAs, created with
 * sto_group_create_ex), g's lanes on the others, all over the same input
 * series u (T x n_in, host or device; b and every member of g must have the
 * same n_in, and the same device).  The sweep runs its current tile width,
 * ring depth and group count with 512 threads per CTA (autotuned first if it
 * has no plan), on as many of its SMs as balance its tiles; its plan for
 * sto_run_batched is left as it was.  Each part gives the same bits as its
 * own call (sto_run_batched, sto_group_run).
 *   sweep_states_out  T x R x N float32 (host or device) or NULL.
 *   group_states_out  NULL, or n pointers (T x N_i, host or device, or NULL).
 * Errors: STO_EINVAL, STO_ENOTSUP (no SM left for the sweep, a member
 *         re-planned since the group was made, shared memory), STO_ENOMEM,
 *         STO_ETIMEOUT, STO_ECUDA. */
STO_API int sto_run_sweep_group(sto_batch* b, sto_group* g, const float* u, int64_t T, float* sweep_states_out,
                                float* const* group_states_out);

/* Launch plan of the sweep kernel. */
typedef struct {
  int32_t tile_n;              /* reservoirs per tile (BN): MMA N = 2 BN (hi and lo terms), multiple of 16 */
  int32_t slots;               /* depth of the shared-memory copy ring */
  int32_t grid;                /* CTAs of the persistent launch */
  int32_t tiles;               /* 128-oscillator x BN-reservoir tiles per stage */
  int32_t smem_bytes;          /* dynamic shared memory per CTA */
  int32_t tuned;               /* 1: chosen by timing candidates; 0: set by the caller or none yet */
  int32_t candidates;          /* candidates the autotuner timed */
  float tuned_us_per_stage;    /* the winner's time per stage in the tuning run */
  int32_t staged;              /* 1: the update loads the next pair's state into registers while it
                                  computes the current pair */
  int32_t groups;              /* reservoir groups with their own grid barriers (1 or 2): with 2, one
                                  group's tensor-core product overlaps the other's update */
  int32_t threads;             /* threads per CTA: 512 (12 update warps of 128 registers) or 1024
                                  (28 update warps of 64 registers) */
  int32_t reserved;
} sto_batch_plan;

/* Set the plan: tile_n (multiple of 8 in [16, 128]) and slots (2 to 9 ring
 * slots of two 64-wide K slices each: 2 (16 KB + 256 tile_n B) of shared
 * memory per slot; three copy warps, warp p owning the slots s = p mod 3),
 * with one reservoir group and 512 threads per CTA, or (0, 0) to time every
 * candidate (tile_n in {16, 32, 40, 48, 64, ..., 128} up to R, slots in
 * {2, 3, 4, 5}, the next pair's state loaded ahead or not, 1 and 2 groups,
 * 512 and 1024 threads) on two RK4 steps of zero
 * input from the batch's state (restored afterwards) and keep the fastest.
 * Tuned plans are cached per (device, N, R) for the life of the process.
 * The stage state is kept.
 * Errors: STO_EINVAL, STO_ENOTSUP (plan cannot run: shared memory, tile
 * shape), STO_ENOMEM, STO_ETIMEOUT, STO_ECUDA.  No counterpart in the paper. */
STO_API int sto_batch_set_plan(sto_batch* b, int32_t tile_n, int32_t slots);

/* sto_batch_set_plan with the number of reservoir groups (1 or 2; 2 needs at
 * least two tile columns, i.e. R > tile_n): the tile columns are split into
 * that many groups, each with its own grid barrier, so that with 2 the
 * tensor-core product of one group runs while the other group's update
 * finishes.  (0, 0, any) runs the autotuner.  Errors: as sto_batch_set_plan;
 * STO_EINVAL for groups outside 1..2. */
STO_API int sto_batch_set_plan_ex(sto_batch* b, int32_t tile_n, int32_t slots, int32_t groups);

/* sto_batch_set_plan_ex with the staging mode: staged = 1 loads the next
 * pair's state into registers while the current pair is computed (and the
 * first pair's while the tile's product runs), 0 loads each pair's state
 * when it is needed, -1 chooses (1 with 512 threads).  512 threads per CTA.
 * Errors: as sto_batch_set_plan_ex; STO_EINVAL for staged outside -1..1. */
STO_API int sto_batch_set_plan_staged(sto_batch* b, int32_t tile_n, int32_t slots, int32_t groups,
                                      int32_t staged);

/* sto_batch_set_plan_staged with the threads per CTA: 512 (12 update warps,
 * 128 registers each) or 1024 (28 update warps, 64 registers each).  Lets a
 * caller (or a profiler run) fix exactly the plan the autotuner chose.
 * Errors: as sto_batch_set_plan_staged; STO_EINVAL for other thread counts. */
STO_API int sto_batch_set_plan_threads(sto_batch* b, int32_t tile_n, int32_t slots, int32_t groups,
                                       int32_t staged, int32_t threads);

/* The current plan (all zero before the first run or set_plan). */
STO_API int sto_batch_get_plan(const sto_batch* b, sto_batch_plan* out);

/* FP64 states, R x 3 x N (host or device). */
STO_API int sto_batch_get_state(const sto_batch* b, double* m);

STO_API void sto_batch_destroy(sto_batch* b);

/* Report the launch plan. */
STO_API int sto_get_info(const sto_handle* h, sto_info* out);

/* Release all device memory of the handle (NULL is allowed). */
STO_API void sto_destroy(sto_handle* h);

/* Text for a status code, including the CUDA error text of the most recent
 * STO_ECUDA on the calling thread.  The pointer stays valid until the next
 * call on that thread. */
STO_API const char* sto_strerror(int code);

/* STO_ABI_VERSION of the built library. */
STO_API int sto_abi_version(void);

/* Fault injection for tests of the device-side timeouts.  With cta >= 0,
 * the next sto_run on h makes CTA `cta` never publish its oscillators, so
 * every other CTA's wait for them runs into the timeout and the call returns
 * STO_ETIMEOUT with the handle still usable after sto_set_state.  cta < 0
 * clears it.  Only meaningful when the plan has more than one CTA. */
STO_API int sto_debug_inject_stall(sto_handle* h, int32_t cta);

/* Allocation-free variant of sto_run, for callers that must not allocate
 * device memory: code running under a framework or pool allocator that owns
 * all of the device's memory, real-time loops in which cudaMalloc's implicit
 * device synchronisation is not acceptable, or plug-ins that may only use
 * buffers handed to them.  The paper has no counterpart; it is a deployment
 * convenience.
 *
 * Same stepping as sto_run, but no handle: the caller owns every array, all
 * in device memory of the current device, and the library allocates nothing
 * (no cudaMalloc, cudaFree or allocating library routine).  The inter-CTA
 * exchange buffer and the error word live in a fixed 256 KB + 256 B
 * statically allocated device array inside libsto, present on every device
 * that loads the library until the process exits.
 *   N           1 .. 16384 and a multiple of 4 (larger N: STO_ETOOBIG).
 *   params      as for sto_create.
 *   W           N x N row-major float32, 16-byte aligned, read in place.
 *   w_in        N x n_in float32.
 *   state       3 x N float64 (m^x block, m^y block, m^z block), advanced
 *               in place.
 *   u, T, states_out   as for sto_run (states_out may be NULL).
 *   stream      cudaStream_t to order the work on (NULL = legacy default).
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * Every call reuses the same array, which keeps the previous call's
 * contents; the call clears what must start fresh.  Calls that overlap on
 * the GPU (two streams, two threads) race on the array and must be
 * serialised by the caller.  Every call first scans all of W and w_in for
 * NaN and Inf (4 N^2 + 4 N n_in bytes read, about 0.2 ms at N = 16384) and
 * synchronises `stream` to read that flag, and synchronises it again at
 * the end to read the device error word.  The library cannot see the
 * extents of the caller's arrays: they must hold the sizes above (the
 * Python binding checks them).
 * Errors: STO_EINVAL (pointer not device memory, N not a multiple of 4,
 *         misaligned W), STO_ETOOBIG, STO_ENONFINITE (W or w_in), STO_ETIMEOUT,
 *         STO_ECUDA, STO_ENOTSUP. */
STO_API int sto_run_noalloc(int64_t N, const sto_params* params, const float* W,
                            const float* w_in, double* state, const float* u,
                            int64_t T, float* states_out, void* stream);

/* ------------------------------------------------------------------------
 * Linear readout of the sampled states.  Sec. 1: in reservoir computing
 * only the readout is trained; the paper does not specify it further.  The
 * readout here is linear with a bias, fitted by ridge regression:
 *     Phi_t = [states[t*N + 0 .. N-1], 1]          (row of N + 1 features)
 *     w     = argmin sum_t (Phi_t w - y_t)^2 + beta |w_0 .. w_{N-1}|^2
 *     beta  = beta_rel * trace(Phi^T Phi) / (N + 1) (the bias is not penalised)
 * solved from the normal equations (Phi^T Phi + beta D) w = Phi^T y by a
 * Cholesky factorisation, all on the GPU in FP64 (the states are FP32 and
 * enter exactly).  Each call allocates its scratch (the (N + 2)^2 FP64 Gram
 * matrix, device copies of host inputs) and frees it before returning, and
 * synchronises `stream` (cudaStream_t, NULL = legacy default) once.
 * ------------------------------------------------------------------------ */

/* Fit w on the samples t in [t0, t1).
 *   states    T x N float32 (row t = the states sampled after input sample
 *             t, as sto_run writes them), host or device; only rows
 *             [t0, t1) are read.
 *   y         T float64 targets, host or device (rows [t0, t1) are read).
 *   beta_rel  >= 0 (0: plain least squares).
 *   w_out     N + 1 float64 weights (bias last), host or device.
 * Limits: 1 <= N <= 32768 (STO_ENOTSUP beyond), 0 <= t0 < t1 <= T.
 * Errors: STO_EINVAL, STO_ENOTSUP, STO_ENONFINITE (NaN or Inf in the rows
 *         or targets), STO_ESINGULAR (the system is not positive definite,
 *         e.g. beta_rel = 0 with fewer samples than features), STO_ENOMEM,
 *         STO_ECUDA. */
STO_API int sto_readout_fit(const float* states, int64_t T, int64_t N, const double* y, int64_t t0,
                            int64_t t1, double beta_rel, double* w_out, void* stream);

/* y_hat[t] = sum_k states[t*N + k] w[k] + w[N] for every t in [0, T), in
 * FP64.  states: T x N float32, w: N + 1 float64, y_hat: T float64; each host
 * or device.  Errors: STO_EINVAL, STO_ENOTSUP, STO_ENOMEM, STO_ECUDA. */
STO_API int sto_readout_predict(const float* states, int64_t T, int64_t N, const double* w,
                                double* y_hat, void* stream);

/* Normalised mean squared error of the readout w on the samples [t0, t1):
 *     *nmse = mean_t (y_hat_t - y_t)^2 / var_t(y_t)
 * (population variance over the same samples).  states, w, y as above;
 * nmse is a host pointer.  Errors: STO_EINVAL (also for a constant target),
 * STO_ENOTSUP, STO_ENOMEM, STO_ECUDA. */
STO_API int sto_readout_nmse(const float* states, int64_t T, int64_t N, const double* w, const double* y,
                             int64_t t0, int64_t t1, double* nmse, void* stream);

/* ------------------------------------------------------------------------
 * One reservoir split across GPUs by rows.  The coupling of Eq. (coup) is
 * the matrix-vector product W m^x (Sec. 3.3): the GPU that holds rows
 * [row0, row0 + rows) of W advances exactly those oscillators, and per RK4
 * stage needs only the stage values m^x of all N oscillators, which the
 * GPUs exchange between stages (an all-gather of N floats; the caller's
 * collective, e.g. NCCL, on the same stream).  A run is
 *     sto_shard_publish(own x) ; all-gather into x
 *     for every input sample t, RK4 step j < substeps, stage s < 4:
 *         sto_shard_stage(x, s, u_t, flags, own x', states_row) ; all-gather x' into x
 * with flags = STO_SHARD_SAMPLE_START at (j = 0, s = 0) and
 * STO_SHARD_SAMPLE_END at (j = substeps - 1, s = 3).  Results equal those
 * of sto_run on the whole reservoir up to the order of the FP32 row sums
 * (the same double-float torque and RK4 combination).
 * ------------------------------------------------------------------------ */
typedef struct sto_shard sto_shard; /* opaque */

#define STO_SHARD_SAMPLE_START 1  /* form the input field of the block from u_t first */
#define STO_SHARD_SAMPLE_END 2    /* write the sampled component after stage 3 */

/* Create the block [row0, row0 + rows) of a reservoir of N oscillators on the
 * current device.
 *   params     as for sto_create (the same on every block).
 *   W_rows     rows x N float32 (rows row0 .. row0 + rows - 1 of W), host or
 *              device; copied.
 *   w_in_rows  rows x n_in float32, host or device; copied.
 *   m0_rows    3 x rows float32 (m^x block, m^y block, m^z block of these
 *              oscillators), host or device, or NULL for Eq. (initial).
 *   stream     cudaStream_t of every launch of the block.
 * Errors: STO_EINVAL (sizes: 0 <= row0, 1 <= rows, row0 + rows <= N),
 *         STO_ENONFINITE, STO_ENOTSUP, STO_ENOMEM, STO_ECUDA. */
STO_API int sto_shard_create(int64_t N, int64_t row0, int64_t rows, const sto_params* params,
                             const float* W_rows, const float* w_in_rows, const float* m0_rows,
                             void* stream, sto_shard** out);

/* Write the block's stage values for the first stage of a run (m^x of the
 * current state, FP32) to x_rows (rows floats, device).  Asynchronous.
 * Errors: STO_EINVAL, STO_ECUDA. */
STO_API int sto_shard_publish(sto_shard* h, float* x_rows);

/* Finish RK4 stage `stage` (0..3) for the block and write its next stage
 * values to x_next (rows floats, device).
 *   x           the stage values m^x of all N oscillators in oscillator order
 *               (device, 16-byte aligned; entries past N are ignored).
 *   u_t         the input sample (n_in floats, device); read only with
 *               STO_SHARD_SAMPLE_START (allowed at stage 0 only).
 *   flags       STO_SHARD_SAMPLE_START | STO_SHARD_SAMPLE_END (stage 3 only).
 *   states_row  rows floats (device) or NULL: the sampled component after
 *               stage 3 when STO_SHARD_SAMPLE_END is set.
 * One kernel launch on the block's stream; no synchronisation, no waits on
 * other blocks.  Errors (argument checks only): STO_EINVAL, STO_ECUDA. */
STO_API int sto_shard_stage(sto_shard* h, const float* x, int32_t stage, const float* u_t, int32_t flags,
                            float* x_next, float* states_row);

/* The block's state, 3 x rows doubles (host or device).  Synchronises.
 * Errors: STO_EINVAL, STO_ENONFINITE (set), STO_ENOMEM, STO_ECUDA. */
STO_API int sto_shard_set_state_f64(sto_shard* h, const double* m);
STO_API int sto_shard_get_state_f64(const sto_shard* h, double* m);

/* Release the block (NULL is allowed). */
STO_API void sto_shard_destroy(sto_shard* h);

#ifdef __cplusplus
}
#endif

#endif /* STO_H_ */

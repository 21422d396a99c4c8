/*
 * opo.h -- C ABI of libopo.so, a GB300 (sm_103a) implementation of the hot
 * path of an optical parametric oscillator (OPO) simulator after
 * arXiv 2410.02532 ("cuOPO").
 *
 * What one round trip computes (the paper's method):
 *   entry ........ the intracavity pump is replaced by the input pump
 *                  (Sec. 4.1, pump read-in kernel), or, in a pump-resonant
 *                  cavity (TRO, Sec. 4.2), the input pump is added to the
 *                  circulating one; a non-resonant signal/idler restarts from
 *                  zero (Sec. 2.1, boundary conditions apply to resonant
 *                  fields only)
 *   crystal pass . (per crystal, in order, when several are set) nz fixed
 *                  steps of the symmetrized split-step Fourier
 *                  method N/2 - L - N/2 (Sec. 2.2, Eq. (expon)) on the
 *                  coupled-wave equations (Sec. 2.1, Eqs. (CEp)-(CEi));
 *                  linear operator of Eq. (linearop) in the frequency domain,
 *                  nonlinear part by one RK4 step of dz/2 per half step
 *   observables .. output-coupled power per field and the signal spectral
 *                  centroid of this round trip
 *   cavity ....... on resonant fields: intracavity GDD and timing mismatch in
 *                  the frequency domain (Sec. 2.3 item 1), then the mirror
 *                  sqrt(1 - theta) e^{i delta} (Sec. 2.1, Eq. (BC)), then the
 *                  phase modulator (Sec. 2.3 item 2), in the order of the
 *                  main-loop listing of Sec. 4.1
 *
 * Conventions (where the paper is silent; every one is fixed by a test):
 *   - grid: N points over the window T = t_rt, dt = T/N, dnu = 1/T
 *     (Sec. 2.4); tau_n = (n - N/2) dt; Omega_k = 2 pi k'/T with k' = k for
 *     k < N/2 and k - N otherwise;
 *   - DFT X_k = sum_n A_n e^{-2 pi i k n/N}, so d/dtau <-> +i Omega;
 *   - linear step factor per dz:
 *       D_x = exp{dz [-alpha_x/2 + i(-dbeta1_x Omega + beta2_x Omega^2/2
 *                                    - beta3_x Omega^3/tod_div)]},
 *     with dbeta1_x = 1/nu_x - 1/nu_s (a slower field moves to later tau) and
 *     tod_div = 6 (Taylor; the paper prints 3, reachable through tod_div);
 *   - fourth-order dispersion adds i beta4_x Omega^4/24 to the exponent of
 *     D_x; a Kerr index n2 adds self- and cross-phase modulation (cross
 *     terms counted twice) to the nonlinear step;
 *   - two-field (degenerate) mode: dA_p/dz = i (kappa_p/2) A_s^2 e^{-i dk z},
 *     dA_s/dz = i kappa_s A_p A_s* e^{+i dk z};
 *   - kappa_x = 2 pi d_eff / (n_x lambda_x); power P = mean|A|^2 n eps0 c/2
 *     times pi w0^2;
 *   - EOM phase beta sin(2 pi frac(f_pm (tau_n + m t_rt))) at round trip m;
 *   - timing mismatch: resonant spectra times e^{-i Omega delay_s} per round
 *     trip (a positive delay moves the field to later tau).
 *
 * Field index: 0 = pump, 1 = signal, 2 = idler (two-field mode: 0, 1).
 * Units are SI.  Host arrays of complex values are interleaved (re, im)
 * doubles; the caller owns every host buffer, the library copies inputs and
 * writes outputs into caller buffers and owns all device memory of a context.
 *
 * Errors: every entry point returns an opo_status and never aborts or exits.
 * Work is enqueued on the context's stream; device-side errors (non-finite
 * fields) surface as OPO_E_NONFINITE at the next synchronizing call
 * (opo_run_roundtrips with stats, opo_get_fields, opo_get_trace, opo_sync).
 * A context is not thread-safe; distinct contexts may be used from distinct
 * threads.
 */
#ifndef OPO_H
#define OPO_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define OPO_API __attribute__((visibility("default")))
#else
#define OPO_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct opo_ctx opo_ctx;     /* opaque, library-owned */
typedef struct opo_batch opo_batch; /* opaque, library-owned */

typedef enum {
    OPO_OK = 0,
    OPO_E_INVALID = 1,     /* bad argument (null pointer, size, range, non-finite value) */
    OPO_E_NOMEM = 2,       /* device allocation failed */
    OPO_E_CUDA = 3,        /* a CUDA runtime call failed (no device, launch failure ...) */
    OPO_E_NONFINITE = 4,   /* a field became NaN/Inf (dz too large, Sec. 2.4) */
    OPO_E_TIMEOUT = 5,     /* reserved: a bounded device wait gave up */
    OPO_E_STATE = 6,       /* call out of order (crystal or cavity not set) */
    OPO_E_UNSUPPORTED = 7  /* valid request the chosen path cannot run */
} opo_status;

enum { OPO_FP64 = 0, OPO_FP32_PH64 = 1 };               /* opo_grid.precision */
/* Input pump: CW; sech^2 pulse per round trip; a user profile per round
 * trip; or the ns-pulsed regime (Sec. 4.2), a Gaussian in intensity much
 * longer than a round trip, A(t) = A0 exp(-2 ln 2 (t - t0)^2 / fwhm^2), read
 * at t = m t_rt + tau_n in round trip m. */
enum { OPO_PUMP_CW = 0, OPO_PUMP_SECH2 = 1, OPO_PUMP_USER = 2, OPO_PUMP_NS = 3 };
enum { OPO_INTRACAVITY = 0, OPO_OUTPUT = 1 };           /* opo_get_fields which */
#define OPO_MAX_CRYSTALS 8  /* crystals per round trip (opo_set_crystals) */
enum { OPO_PATH_AUTO = 0, OPO_PATH_PLAIN = 1, OPO_PATH_FUSED = 2 };

/* Grid and numerics of one OPO instance (Sec. 2.4). */
typedef struct {
    int32_t n;           /* points N: power of two in [16, 131072]                 */
    double  t_window_s;  /* window T = t_rt [s], > 0                               */
    int32_t nfields;     /* 3 (pump, signal, idler) or 2 (degenerate)              */
    int32_t precision;   /* OPO_FP64: all FP64.  OPO_FP32_PH64: FP32 complex
                            fields, phase arguments formed in FP64 and rounded
                            once                                                    */
    int32_t device;      /* CUDA device ordinal                                     */
    void   *stream;      /* cudaStream_t to enqueue on; NULL: the context makes a
                            private non-blocking stream                            */
} opo_grid;

/* Nonlinear crystal (Sec. 2.1).  Triples are indexed by field. */
typedef struct {
    double  length_m;           /* L > 0                                           */
    int32_t nz;                 /* fixed z-steps per pass, >= 1                    */
    double  dk_per_m;           /* Delta k = k_p - k_s - k_i                       */
    double  deff_mpv;           /* d_eff [m/V]                                     */
    double  lambda_m[3];        /* vacuum wavelengths, > 0 for used fields         */
    double  n[3];               /* refractive indices, > 0 for used fields         */
    double  alpha_per_m[3];     /* power attenuation                               */
    double  dbeta1_s_per_m[3];  /* 1/nu_x - 1/nu_s                                 */
    double  beta2_s2_per_m[3];  /* GVD k''                                         */
    double  beta3_s3_per_m[3];  /* TOD k'''                                        */
    double  w0_m;               /* beam waist for power <-> intensity, > 0         */
    double  tod_div;            /* divisor of the TOD term; 0 selects 6            */
    /* extensions the paper names without equations (Sec. 1, Sec. 2.1):      */
    double  beta4_s4_per_m[3];  /* fourth-order dispersion: i beta4 Omega^4/24 in
                                   the exponent of D_x                              */
    double  n2_m2_per_W;        /* Kerr index: dA_x/dz += i (2 pi/lambda_x) n2
                                   (I_x + 2 sum_{y != x} I_y) A_x, I_y =
                                   n_y eps0 c |A_y|^2 / 2; 0 = no chi(3) terms     */
} opo_crystal;

/* Cavity and pump (Sec. 2.1 Eq. (BC), Sec. 2.3, Sec. 4). */
typedef struct {
    uint32_t resonant_mask;  /* bit x: field x resonant (SRO/DRO/TRO, Sec. 4.2)    */
    double  R[3];            /* mirror power reflectivity 1 - theta_x, in [0, 1]   */
    double  delta_rad[3];    /* detuning phase delta_x (Eq. (BC))                  */
    double  gdd_s2[3];       /* intracavity GDD gamma_x [s^2] (Sec. 2.3 item 1)    */
    double  delay_s;         /* per-round-trip timing mismatch of resonant fields  */
    double  eom_beta_rad;    /* EOM depth beta (Sec. 2.3 item 2); 0 = no EOM       */
    double  eom_f_hz;        /* EOM frequency f_pm                                 */
    double  t_rt_s;          /* round-trip time in the EOM phase; 0 = t_window_s   */
    int32_t pump_kind;       /* OPO_PUMP_CW / _SECH2 / _USER / _NS                  */
    double  pump_power_W;    /* CW power, or sech^2 / ns-pulse peak power          */
    double  pump_fwhm_s;     /* sech^2 or ns-pulse intensity FWHM, > 0 for those   */
    const double *pump_user; /* OPO_PUMP_USER: 2N interleaved doubles [V/m], copied */
    double  pump_t0_s;       /* OPO_PUMP_NS: pulse centre t0 on the axis m t_rt +
                                tau_n (t_rt as for the EOM)                        */
} opo_cavity;

/* Result of opo_run_roundtrips (filled only when a pointer is passed, which
 * synchronizes the stream). */
typedef struct {
    int64_t rt_done;          /* round-trip counter m after the call               */
    double  p_out_W[3];       /* output-coupled power per field, last round trip   */
    double  centroid_hz;      /* signal spectral centroid, last round trip         */
    double  p_out_mean_W[3];  /* mean over the last max(10, ceil(M/10)) round trips */
    double  centroid_mean_hz; /* of this call (all of them if M < 10)              */
    int32_t path;             /* OPO_PATH_PLAIN or OPO_PATH_FUSED                  */
    int32_t cluster;          /* CTAs per instance of the fused path (0: plain)    */
} opo_stats;

/* Check a configuration without touching any GPU: the grid as opo_create
 * checks it (apart from the device ordinal), `count` crystals as
 * opo_set_crystals checks them (count 0: none; crystals may then be NULL)
 * and the cavity as opo_set_cavity checks it (NULL: none).  Returns OPO_OK
 * or OPO_E_INVALID.  The context calls run the same checks. */
OPO_API int opo_validate(const opo_grid *grid, const opo_crystal *crystals, int32_t count,
                         const opo_cavity *cavity);

/* Create a context for one OPO instance on grid->device.  Fields start at
 * zero; a zero signal never grows, so seed it with opo_set_fields.
 * Returns OPO_E_INVALID for a bad grid, OPO_E_CUDA if the device is missing,
 * OPO_E_NOMEM if allocation fails.  *out is NULL on failure. */
OPO_API int opo_create(opo_ctx **out, const opo_grid *grid);

/* Set the crystal (Sec. 2.1); rebuilds the per-step dispersion factors D_x
 * (FP64 arguments, one rounding) on the device.  Copies *crystal. */
OPO_API int opo_set_crystal(opo_ctx *ctx, const opo_crystal *crystal);

/* Several nonlinear crystals per round trip (the paper notes that one or
 * more nonlinear media can be placed in the cavity): count in
 * [1, OPO_MAX_CRYSTALS] crystals, passed in array order every round trip.
 * The fields go on unchanged from one crystal to the next (no interface or
 * free-space step between them) and z of the e^{i dk z} factor restarts at 0
 * in each.  Every crystal keeps its own length, steps, dk, d_eff, indices,
 * loss, dispersion and Kerr index; lambda_m must be the same in all of them
 * (the same fields), and the input pump amplitude and the output powers use
 * crystals[0]'s indices and waist.  opo_set_crystal(ctx, k) is
 * opo_set_crystals(ctx, k, 1).  OPO_E_INVALID for a bad count, a bad crystal
 * or differing wavelengths.  Copies the array. */
OPO_API int opo_set_crystals(opo_ctx *ctx, const opo_crystal *crystals, int32_t count);

/* Set the cavity and pump (Eq. (BC), Sec. 2.3); rebuilds the input pump, GDD
 * and delay factors on the device.  Copies *cavity and pump_user. */
OPO_API int opo_set_cavity(opo_ctx *ctx, const opo_cavity *cavity);

/* Copy n complex values (2n interleaved doubles) into intracavity field
 * `field`; n must equal the grid's N.  rt_index >= 0 also sets the
 * round-trip counter m (the EOM phase depends on it) and clears a pending
 * non-finite error (a new start); -1 leaves both. */
OPO_API int opo_set_fields(opo_ctx *ctx, int32_t field, const double *interleaved, size_t n,
                   int64_t rt_index);

/* Run m >= 0 round trips, enqueued on the context's stream.  stats may be
 * NULL (no synchronization); otherwise the call waits and fills it.
 * OPO_E_STATE before both opo_set_crystal and opo_set_cavity. */
OPO_API int opo_run_roundtrips(opo_ctx *ctx, int64_t m, opo_stats *stats);

/* Copy field `field` into out (2n doubles, n = N).  which = OPO_INTRACAVITY:
 * the state that starts the next round trip; OPO_OUTPUT: the output-coupled
 * field sqrt(1 - R_x) A_x (resonant) or A_x (non-resonant) of the last round
 * trip, zero before the first.  Synchronizes the stream. */
OPO_API int opo_get_fields(opo_ctx *ctx, int32_t field, int32_t which, double *out, size_t n);

/* Output history, the per-round-trip output vectors the paper saves (e.g.
 * the output pump and signal of an ns pulse over its round trips, Sec. 4.2):
 * with max_rt > 0 every following opo_run_roundtrips / opo_batch_run call
 * records the output-coupled fields of each of its round trips, row r of the
 * history holding round trip r of the call (F x N complex values in the
 * context's precision, on the device).  max_rt = 0 frees the history.
 * While it is on, a call with more than max_rt round trips returns
 * OPO_E_INVALID.  OPO_E_NOMEM if the rows cannot be allocated. */
OPO_API int opo_set_output_history(opo_ctx *ctx, int64_t max_rt);

/* Copy rows [row0, row0 + rows) of field `field` of the output history into
 * out (rows x 2N doubles, interleaved re/im).  OPO_E_STATE without a history;
 * OPO_E_INVALID for rows outside it.  Synchronizes. */
OPO_API int opo_get_output_history(opo_ctx *ctx, int32_t field, int64_t row0, int64_t rows,
                                   double *out);

/* Copy the per-round-trip observables of the last opo_run_roundtrips call:
 * rows {P_p_out, P_s_out, P_i_out, nu_c} [W, W, W, Hz], `rows` rows (at most
 * the call's M).  Synchronizes. */
OPO_API int opo_get_trace(opo_ctx *ctx, double *out, int64_t rows);

/* Device-resident variants for callers that keep fields on the GPU (for
 * example in torch tensors): dev points to n complex values in the
 * context's precision (float2 or double2 interleaved) on the context's
 * device.  Stream-ordered; no synchronization. */
OPO_API int opo_set_fields_device(opo_ctx *ctx, int32_t field, const void *dev, size_t n,
                          int64_t rt_index);
OPO_API int opo_get_fields_device(opo_ctx *ctx, int32_t field, int32_t which, void *dev, size_t n);

/* Choose the execution path.  OPO_PATH_PLAIN: one kernel per operation per
 * z-step, replayed as a CUDA graph per round trip.  OPO_PATH_FUSED: one
 * persistent kernel per launch in which a thread-block cluster of `cluster`
 * CTAs of `threads` threads keeps the instance's fields in distributed shared
 * memory for `rt_per_launch` round trips.  0 picks the default for each of
 * cluster, rt_per_launch and threads; the default shapes favour batches
 * (where two CTAs fit an SM's shared memory, CTAs small enough that the
 * registers admit two as well), and a lone instance may run faster with
 * larger CTAs.  OPO_E_UNSUPPORTED if the fused path cannot hold the instance
 * in that configuration. */
OPO_API int opo_set_path(opo_ctx *ctx, int32_t path, int32_t cluster, int32_t rt_per_launch,
                         int32_t threads);

/* Fused-path capacity on the context's device: how many thread-block
 * clusters of `cluster` CTAs (0: the default size for this instance) with
 * this instance's shared-memory footprint can be resident at once, i.e. how
 * many such instances one batched launch runs concurrently (threads = 0: the
 * default CTA size).  *cluster_out
 * (optional) receives the cluster size used.  OPO_E_UNSUPPORTED if the fused
 * path cannot hold the instance. */
OPO_API int opo_fused_capacity(const opo_ctx *ctx, int32_t cluster, int32_t threads,
                               int32_t *max_active, int32_t *cluster_out);

/* Wait for the context's stream; reports a pending device error. */
OPO_API int opo_sync(opo_ctx *ctx);

/* Free the context and its device memory (NULL is accepted). */
OPO_API int opo_destroy(opo_ctx *ctx);

/* Static string for a status code. */
OPO_API const char *opo_status_string(int status);

/* Batched sweep: many instances advanced together.  A member whose
 * opo_set_path asks for the fused path, or leaves the choice to the library
 * (OPO_PATH_AUTO) at a size the fused kernels hold, runs on the fused path,
 * one thread-block cluster per instance; these are grouped by (N, field
 * count, nonlinear-step kernel variant: chi(2) with a phase mismatch in some
 * crystal, chi(2) with dk = 0 in all, or with Kerr terms, and launch shape),
 * each group one persistent launch.  The other members run on the plain path
 * (one kernel per operation, Sec. 2.2 and the main loop of Sec. 4.1), grouped
 * by (N, field count, the crystals' step counts): every launch of a group
 * applies one operation to all of its members, and one round trip of the
 * group is a captured graph.  The groups run concurrently.  A member whose
 * crystals or path request change after opo_batch_create so that it no
 * longer fits its group makes opo_batch_run return OPO_E_STATE (make a new
 * batch).  All contexts must be on one device, in one precision, with
 * crystal and cavity set; every other parameter may differ.  The batch keeps
 * pointers to the contexts (owned by the caller; they must outlive the batch)
 * and is ordered on the first context's stream.  opo_batch_run needs every
 * member alive; opo_batch_destroy does not read the members (it waits for the
 * device), so a batch may be destroyed after or before its contexts.  Each instance advances
 * bit-for-bit as opo_run_roundtrips would advance it alone on the same path
 * with the same launch shape: `cluster` and `threads` apply to every
 * instance when nonzero; where zero, each instance keeps the cluster size,
 * CTA size and round trips per launch of its own opo_set_path (default 0:
 * the library's choice for its size class).
 * OPO_E_UNSUPPORTED if a member that asks for the fused path cannot run with
 * that cluster size. */
OPO_API int opo_batch_create(opo_batch **out, opo_ctx *const *ctxs, int32_t count, int32_t cluster,
                             int32_t threads);
OPO_API int opo_batch_run(opo_batch *batch, int64_t m);

/* on = 1: run every fused member of the batch in one persistent launch (the
 * batched sweep of mixed sizes as a single kernel launch): one cluster size
 * and CTA size for all, those that hold the largest member, and the generic
 * fused kernel when sizes or field counts differ (it takes N, F and every
 * parameter per instance from its descriptor).  The launch configuration
 * then follows the largest member, so a member's rounding may depend on the
 * mix (and differ from its lone run, which uses its size class's own
 * kernel); results stay within the stated tolerances of the oracle.  on = 0:
 * one launch per size class again (the default: each class keeps its own
 * kernel, cluster and CTA size, and every member advances bit for bit as it
 * would alone).  Plain-path members are not affected.  OPO_E_UNSUPPORTED if
 * no single configuration holds every fused member.  Waits for the device. */
OPO_API int opo_batch_set_one_launch(opo_batch *batch, int32_t on);
OPO_API int opo_batch_destroy(opo_batch *batch);

/* Host transfers of a whole batch (one copy each way instead of one per field
 * and instance).  opo_batch_set_fields: `host` holds every member's F x N
 * complex start state, members in batch order, fields in order, interleaved
 * re/im doubles; count = sum over members of F N (OPO_E_INVALID otherwise).
 * The round-trip counters are not touched; the host buffer is free to reuse
 * when the call returns.  opo_batch_get_fields: field `field` (INTRACAVITY or
 * OUTPUT, as opo_get_fields) of every member into host, members in order, N
 * complex each (zeros for a member without that field); count = sum of N.
 * opo_batch_get_trace: the first `rows` trace rows of the last call of every
 * member, members in order, rows x 4 doubles each (rows at most the last
 * call's round trips).  Both getters synchronize and return OPO_E_NONFINITE
 * if any member holds a non-finite field. */
OPO_API int opo_batch_set_fields(opo_batch *batch, const double *host, size_t count);
OPO_API int opo_batch_get_fields(opo_batch *batch, int32_t field, int32_t which, double *host,
                                 size_t count);
OPO_API int opo_batch_get_trace(opo_batch *batch, double *host, int64_t rows);

/* One step of a batch with its host transfers in flight beside the other
 * steps' round trips: the main loop of Sec. 4.1 (fields in, round trips,
 * output fields and observables out) for a stream of batch steps.  The call
 * only enqueues work and returns:
 *   1. host_in (if not NULL: every member's F x N start state, layout and
 *      count as opo_batch_set_fields; page-locked host memory) is copied to a
 *      device staging slot on a copy stream of the batch, so that the copy
 *      overlaps the previous step's round trips, then written into the
 *      members' fields in stream order;
 *   2. m round trips of every member (as opo_batch_run);
 *   3. if host_out is not NULL: field `field` of every member's output
 *      (OPO_OUTPUT, layout as opo_batch_get_fields, sum of N complex) and
 *      then the last trace row of every member (4 doubles each, members in
 *      order) are gathered into a device slot and copied to host_out on a
 *      second copy stream, so that the copy overlaps the next step.
 * Two staging slots alternate between consecutive calls.  host_in must not
 * change, and host_out must not be read, until opo_batch_io_wait returns;
 * consecutive calls may reuse the same host buffers.  opo_batch_io_wait
 * waits for every enqueued step and copy of the batch and returns
 * OPO_E_NONFINITE if any member holds a non-finite field.  Errors of the
 * arguments return before anything is enqueued (OPO_E_INVALID; m >= 1;
 * 0 <= field < the members' least field count). */
OPO_API int opo_batch_step_io(opo_batch *batch, const double *host_in, double *host_out,
                              int32_t field, int64_t m);
OPO_API int opo_batch_io_wait(opo_batch *batch);

/* One crystal pass without any device allocation, for callers that cannot
 * call cudaMalloc (code that runs inside another framework's memory pool or
 * under an allocator that is locked down or already exhausted).  The paper
 * has no counterpart; it is the crystal pass of opo_run_roundtrips (plain
 * path) without a context.
 *
 * fields: device pointer to grid->nfields x grid->n complex values in the
 *         grid's precision (float2 for OPO_FP32_PH64, double2 for OPO_FP64),
 *         field-major, advanced in place by crystal->nz symmetrized steps.
 * stream: cudaStream_t to enqueue on (NULL = legacy default stream); the call
 *         returns without synchronizing; grid->stream is ignored.
 * Scratch: a fixed 4 MiB device array inside the library, shared by every
 *         call on a device and held by every GPU that loads the library until
 *         the process exits.  It needs
 *         bytes(c) = round256(c N) + 2 round256(c F N) + round256(c (4 nz + 1))
 *         <= 4 MiB with c = 8 (FP32) or 16 (FP64), e.g. N <= 2^15 with 3
 *         fields in FP64, N <= 2^16 in FP32; larger requests return
 *         OPO_E_INVALID without launching anything.  Every call rewrites all
 *         of the scratch it reads (nothing must start at zero).  Calls whose
 *         work overlaps on the GPU (other streams, other threads) race on the
 *         shared scratch: serialize them.
 * Set-up: every call looks up the array's device address with that device
 *         current (a lookup, no allocation; the first one on a device may
 *         load the library's device code, so make it before any stream
 *         capture). */
OPO_API int opo_crystal_pass_noalloc(const opo_grid *grid, const opo_crystal *crystal,
                                     void *fields, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* OPO_H */

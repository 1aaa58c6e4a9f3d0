/*
 * rr.h -- C ABI of the GB300 (sm_103a) RoadRunner transit light-curve library.
 *
 * RoadRunner (Parviainen 2020, MNRAS) evaluates a transit light curve as
 * Eq. 5:  f = (I_star - (w . l) a(c, k)) / I_star,
 * where a(c, k) is the area of the stellar disk covered by a planet of
 * radius ratio k at projected centre distance c, w . l the mean covered
 * brightness (a weight vector over radial annuli dotted with the limb-
 * darkening profile l, Sect. 2), and I_star the disk-integrated brightness
 * (Eq. 2-4).  The weights are tabulated on a (k, g) grid, g = c / (1 + k),
 * and interpolated (Sect. 3.1, 3.1.2).  Each light-curve point is the mean
 * of f over exposure sub-samples (Sect. 4.1); the planet's distance comes
 * from a Keplerian orbit with the parameters of Sect. 4.1.
 *
 * Conventions for every entry point:
 *  - Device pointers are CUDA device memory on the context's device, host
 *    pointers ordinary host memory.  Each argument says which.  The caller
 *    owns every pointer it passes; the library keeps none of them after
 *    the call returns (host arrays are copied).
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  rr_evaluate / rr_evaluate_grad only enqueue work: results
 *    are valid once the stream has been synchronised.
 *  - Argument errors are detected on the host before anything is enqueued
 *    and return a non-zero rr_status; rr_last_error() then describes it.
 *  - A parameter vector (pv) outside the model's domain does not fail the
 *    call: its light curve is NaN and its pv_status word is non-zero
 *    (RR_PV_* bits below).
 *  - A context is not thread-safe: calls on one context must not overlap
 *    in time on the host.  Distinct contexts are independent.  Evaluations
 *    on different streams may overlap on the device if each has its own
 *    workspace and output buffers.
 */
#ifndef RR_H
#define RR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rr_ctx rr_ctx;

typedef enum {
    RR_OK = 0,
    RR_EINVAL = 1,    /* bad argument (null pointer, size, range, layout) */
    RR_ENOMEM = 2,    /* device or host allocation failed */
    RR_ECUDA = 3,     /* a CUDA runtime call or kernel launch failed */
    RR_ESTATE = 4,    /* call out of order (e.g. evaluate before rr_build_weights) */
    RR_EDOMAIN = 5,   /* a requested accuracy cannot be met (rr_choose_grid) */
    RR_ETIMEOUT = 6,  /* a bounded device-side wait gave up (see rr_last_error) */
    RR_EPAGEABLE = 7  /* a host buffer given to the server is not page-locked */
} rr_status;

/* Limb-darkening laws (Sect. 3.2.1, in their usual forms; all affine in their
 * coefficients, with closed-form disk integrals) and the tabulated numerical
 * profile (Sect. 3.2.2). */
typedef enum {
    RR_LD_UNIFORM = 0,        /* I = 1                                      0 coefficients */
    RR_LD_QUADRATIC = 1,      /* I = 1 - u1 (1-mu) - u2 (1-mu)^2            2 (u1, u2)     */
    RR_LD_QUADRATIC_TRI = 2,  /* quadratic with u1 = 2 sqrt(q1) q2,
                                 u2 = sqrt(q1) (1 - 2 q2) (Kipping)         2 (q1, q2)     */
    RR_LD_NONLINEAR = 3,      /* I = 1 - sum_n c_n (1 - mu^(n/2)), n=1..4   4 (c1..c4)     */
    RR_LD_TABULATED = 4,      /* I(mu) given per passband by rr_set_ld_profile   0        */
    RR_LD_LINEAR = 5,         /* I = 1 - u (1-mu)                           1 (u)          */
    RR_LD_GENERAL = 6,        /* I = 1 - sum_n c_n (1-mu)^n, n=1..N         N = rr_config.ncoef, 1..4 */
    RR_LD_LOGARITHMIC = 7,    /* I = 1 - u1 (1-mu) - u2 mu ln(mu)           2 (u1, u2)     */
    RR_LD_EXPONENTIAL = 8,    /* I = 1 - u1 (1-mu) - u2 / (1 - exp(mu))     2 (u1, u2)     */
    RR_LD_POWER2 = 9,         /* I = 1 - c (1 - mu^alpha), alpha > 0        2 (c, alpha)   */
    RR_LD_POWER2_PM = 10      /* power-2 with h1 = I(1/2), h2 = I(1/2) - I(0):
                                 c = 1 - h1 + h2, alpha = log2(c / h2)      2 (h1, h2)     */
    /* The power-2 laws are not affine in alpha, so no weight projection can be
     * tabulated for them: they need the direct model (rr_config.direct = 1),
     * which forms the profile of every pv inside its per-call weight pass, and
     * they do not combine with the small-planet approximation. */
} rr_ld_model;

typedef enum {
    RR_PREC_FP64 = 0,   /* every step in FP64; flux and grad_flux are double */
    RR_PREC_MIXED = 1   /* FP64 setup, phase reduction and normalisation; FP32 bulk;
                           flux and grad_flux are float.  Flux within 1e-6 absolute
                           of the FP64 form (Kepler in FP64 above e = 0.8) */
} rr_precision;

/* Per-pv status bits written to pv_status (0 = valid). */
#define RR_PV_K_RANGE    1    /* a radius ratio outside (0, 1), or the weights' radius ratio outside
                                 [k0, k1] (interpolated model, not below k_small) */
#define RR_PV_E_RANGE    2    /* eccentricity outside [0, 1) */
#define RR_PV_B_RANGE    4    /* impact parameter outside [0, a] */
#define RR_PV_P_RANGE    8    /* period <= 0 */
#define RR_PV_NONFINITE  16   /* a non-finite parameter */
#define RR_PV_LD_INVALID 32   /* I_star <= 0, or q1/q2 outside [0, 1] */
#define RR_PV_A_RANGE    64   /* scaled semi-major axis <= 1 */
#define RR_PV_KEPLER     128  /* Kepler iteration did not converge at some point (NaN there) */

#define RR_MAX_PB 32          /* passbands per context */

typedef struct {
    double  zcut;       /* radial grid split, 0 < zcut < 1 (Sect. 3.1.1) */
    int32_t nzin;       /* annuli of constant dz inside zcut, >= 1 */
    int32_t nzlimb;     /* annuli of constant dmu outside zcut, >= 1; nz = nzin + nzlimb <= 4096 */
    int32_t ng;         /* grazing-value nodes g_i = i / (ng - 1), 2 <= ng <= 4096 */
    int32_t nk;         /* radius-ratio nodes on [k0, k1] (Sect. 3.1.2), 2 <= nk <= 4096;
                           unused (not checked) by the direct model */
    double  k0, k1;     /* radius-ratio range, 0 < k0 < k1 < 1; unused by the direct model */
    int32_t npb;        /* passbands, 1 <= npb <= RR_MAX_PB */
    int32_t ld_model;   /* rr_ld_model */
    int32_t chromatic;  /* 0: one k per pv; 1: one k per passband (Sect. 4.2) */
    int32_t precision;  /* rr_precision */
    int32_t device;     /* CUDA device ordinal */
    int32_t ncoef;      /* terms of RR_LD_GENERAL (1..4); 0 for every other law */
    int32_t direct;     /* 0: the interpolated model, weights tabulated on the (k, g) grid and
                           interpolated in k and g (Sect. 3.1.2);
                           1: the direct model of the same section: every call computes the
                           weights on the g grid for each parameter vector's own k, with
                           0 < k < 1 (interpolation in g only; no k table, no k range) */
    int32_t shared_weights; /* transmission spectroscopy (Sect. 3.4), with chromatic = 1: every
                           passband of a pv uses one weight array, computed at the mean of the
                           pv's radius ratios; the area and g = z / (1 + k) keep each passband's
                           own k.  0 = one weight array per passband.  No effect otherwise. */
    double  k_small;    /* small-planet approximation (Sect. 3.4): a passband whose (weights')
                           radius ratio is below k_small uses, at every g node, the profile at
                           the planet's centre, I(mu), mu = sqrt(1 - min(g (1 + k), 1)^2) clamped
                           below to the outermost bin mean, instead of the weighted average; it
                           needs no k table (0 < k < k_small is valid).  0 = off; >= 0, finite. */
} rr_config;

/* Create a context: validates `cfg`, builds the radial grid of Sect. 3.1.1 on
 * the host in FP64 (edges ze, means zm = midpoints, mu = sqrt(1 - zm^2)) and
 * allocates the device tables.  Named LD laws are ready at once; the
 * tabulated law needs rr_set_ld_profile for every passband.  *out receives
 * the context (NULL on failure).  Errors: RR_EINVAL (cfg), RR_ENOMEM, RR_ECUDA. */
rr_status rr_create(const rr_config* cfg, rr_ctx** out);

/* Free the context and all device memory it owns.  Accepts NULL. */
rr_status rr_destroy(rr_ctx* ctx);

/* Set the numerical profile of passband `pb` (Sect. 3.2.2): host arrays mu[n]
 * (strictly increasing, within [0, 1]) and intensity[n] (finite), n >= 2,
 * copied.  Between nodes the profile is linear, outside them constant; its
 * normalisation I_star is the exact integral of that function (Eq. 2).
 * Only for RR_LD_TABULATED.  Invalidates the tables until the next
 * rr_build_weights.  Errors: RR_EINVAL, RR_ESTATE (named law). */
rr_status rr_set_ld_profile(rr_ctx* ctx, int32_t pb, const double* mu, const double* intensity,
                            int32_t n);

/* Build the tables (Sect. 3.1.2): the LD profiles at the bin means and their
 * disk integrals, the FP64 weight table w[nk][ng][nz] (covered annulus area
 * / covered area, Sect. 2), and its projections T[b][nk][ng] = w . l_b onto
 * every profile basis b.  The direct model builds no (k, g) table: it keeps
 * the profiles, their disk integrals and, per basis, the running sums over
 * annuli of (annulus area x profile) that a planet covering the disk's
 * centre takes whole; its weights are computed by every evaluation.
 * Enqueued on `stream`, then the stream is synchronised (set-up, not hot
 * path).  Must precede evaluation.
 * Errors: RR_ESTATE (a tabulated profile missing), RR_ECUDA. */
rr_status rr_build_weights(rr_ctx* ctx, void* stream);

/* Number of columns of a parameter row:
 *   [T0, P, a, b, e, w, k_0 .. k_{nkp-1}, ldc_0 .. ldc_{npb*nldc-1}]
 * T0 = mid-transit (conjunction) time and P = period, in the time unit of
 * `times` (days); a = semi-major axis and b = impact parameter a cos i in
 * stellar radii; e = eccentricity; w = argument of periastron [rad];
 * nkp = npb if chromatic else 1; nldc = coefficients of the LD law, stored
 * passband-major. */
int32_t rr_nparam(const rr_ctx* ctx);

/* Device workspace (bytes) that rr_evaluate (with_grad = 0) or
 * rr_evaluate_grad (with_grad = 1) needs for npv parameter vectors and npt
 * times.  0 on bad arguments. */
size_t rr_workspace_bytes(const rr_ctx* ctx, int32_t npv, int32_t npt, int32_t with_grad);

/* Evaluate light curves: flux[pv][t] for every parameter vector and time --
 * Eq. 5 for each exposure sub-sample, with the mean covered brightness
 * interpolated in (k, g) from the tables of Sect. 3.1.2 (in g only for the
 * direct model), averaged over the sub-exposures of Sect. 4.1; the orbit of
 * the parameters of Sect. 4.1 (Keplerian, conjunction at T0); the passband of
 * each time as in the heterogeneous series of Sect. 4.2.
 *   times        device, double[npt]: mid-exposure times
 *   pb_index     device, int32[npt]: passband of each time, 0 <= . < npb
 *                (NULL allowed when npb == 1)
 *   params       device, double[npv][nparam], row-major (see rr_nparam)
 *   supersampling host, int32[npb]: sub-exposures per time, 1 .. 1024
 *   exptime      host, double[npb]: exposure length, >= 0 (ignored if ss = 1)
 *   flux         device, [npv][npt] row-major, float (MIXED) or double (FP64)
 *   pv_status    device, int32[npv] (RR_PV_* bits), or NULL
 *   workspace    device scratch of >= rr_workspace_bytes(ctx, npv, npt, 0)
 *                bytes, 256-byte aligned; contents are overwritten
 * npt == 0 or npv == 0 is a valid no-op.  Errors: RR_EINVAL, RR_ESTATE, RR_ECUDA. */
rr_status rr_evaluate(rr_ctx* ctx, const double* times, const int32_t* pb_index, int32_t npt,
                      const double* params, int32_t npv, const int32_t* supersampling,
                      const double* exptime, void* flux, int32_t* pv_status, void* workspace,
                      size_t workspace_bytes, void* stream);

/* rr_evaluate without a caller-provided workspace.  The paper has no
 * counterpart: this exists for callers that cannot allocate device memory
 * when they evaluate -- for example code that runs where CUDA allocation
 * calls are not allowed (such as a host function enqueued on a stream), or
 * an application that hands all device memory to its own allocator up front
 * and has none left to lend.  The scratch this call needs (per-pv records
 * and per-time inputs, as counted by rr_workspace_bytes(ctx, npv, npt, 0))
 * lives in a fixed array of RR_NOALLOC_SCRATCH_BYTES inside the library,
 * which every GPU that loads the library holds until the process exits.
 *   - Allocates nothing: no cudaMalloc/cudaFree and no allocating library
 *     routine.  Arguments as rr_evaluate, minus the workspace.
 *   - Batches needing more than RR_NOALLOC_SCRATCH_BYTES are rejected with
 *     RR_EINVAL and a message naming the sizes (split the batch, or use
 *     rr_evaluate with your own workspace).
 *   - All calls in the process share the one array per device: calls whose
 *     work overlaps on the GPU (different streams, or different contexts on
 *     the same device, without ordering between them) race on it and give
 *     wrong results.  Order them, or use rr_evaluate.
 *   - The array keeps the last call's contents; every call rewrites what it
 *     reads before reading it, so nothing needs clearing.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress, with that device made current); make that first
 *     call before any stream capture on that device.  The address is kept
 *     for the life of the process: it does not survive cudaDeviceReset (or
 *     any other teardown of the device's primary context), after which this
 *     entry point must not be called.
 * Errors: as rr_evaluate, plus RR_EINVAL for oversize batches. */
#define RR_NOALLOC_SCRATCH_BYTES (32u << 20)
rr_status rr_evaluate_noalloc(rr_ctx* ctx, const double* times, const int32_t* pb_index, int32_t npt,
                              const double* params, int32_t npv, const int32_t* supersampling,
                              const double* exptime, void* flux, int32_t* pv_status, void* stream);

/* Vector-Jacobian product of rr_evaluate (hand-written adjoint; the paper has
 * no adjoint: this differentiates Eq. 5, the interpolants of Sect. 3.1.2 and
 * the orbit of Sect. 4.1 by the chain rule):
 *   grad_params[pv][j] = sum_t grad_flux[pv][t] * d flux[pv][t] / d params[pv][j]
 * Same inputs as rr_evaluate, plus
 *   grad_flux    device, [npv][npt], float (MIXED) or double (FP64)
 *   grad_params  device, double[npv][nparam] (written, not accumulated)
 * Derivatives of the piecewise-linear (k, g) interpolants are those of the
 * cell holding the point (the lower cell on a node).  The sum over times is
 * deterministic (fixed tiling and order), so a pv's gradient does not
 * depend on the other pvs evaluated with it.  Invalid pvs get NaN rows.
 * Accuracy (MIXED): a component that is a sum of same-sign terms (for
 * example the cotangent sign(d flux / d params[j]) for component j) is
 * within 1e-5 relative of the exact chain rule, 1e-4 for the exponential
 * law (unbounded at the limb); samples near a contact point or a g node are
 * recomputed in float-float for this.  A component that is a cancelling sum
 * carries the absolute error of its terms instead.
 * workspace >= rr_workspace_bytes(ctx, npv, npt, 1).  Errors as rr_evaluate. */
rr_status rr_evaluate_grad(rr_ctx* ctx, const double* times, const int32_t* pb_index, int32_t npt,
                           const double* params, int32_t npv, const int32_t* supersampling,
                           const double* exptime, const void* grad_flux, double* grad_params,
                           int32_t* pv_status, void* workspace, size_t workspace_bytes,
                           void* stream);

/* Shared set-up for one flux evaluation and one adjoint on the same batch
 * (the forward and backward passes of a fit step).  rr_evaluate and
 * rr_evaluate_grad each run the per-pv set-up (orbit constants, transit
 * windows, the k-interpolated profile rows of Sect. 3.1.2 divided by I_star)
 * and the per-time preparation before their main kernel; rr_prepare runs
 * them once, in the adjoint's record layout, into `workspace`, and
 * rr_evaluate_prepared / rr_evaluate_grad_prepared then run only the main
 * kernels.  The paper has no counterpart (its model has no adjoint).
 *   - All three take the arguments of rr_evaluate_grad (minus the outputs
 *     they do not write); the two evaluation calls must be given the same
 *     times, pb_index, params, supersampling, exptime and workspace as the
 *     rr_prepare call, and the workspace must not change in between (the
 *     library cannot check this: different inputs give wrong results).
 *   - workspace: >= rr_workspace_bytes(ctx, npv, npt, 1) bytes, 256-byte
 *     aligned, owned by the caller; it holds the prepared batch until the
 *     caller reuses it.
 *   - pv_status (optional) is written by rr_prepare; the evaluation calls
 *     may add RR_PV_KEPLER.
 *   - Results are bitwise those of rr_evaluate / rr_evaluate_grad.
 * Errors: as rr_evaluate_grad. */
rr_status rr_prepare(rr_ctx* ctx, const double* times, const int32_t* pb_index, int32_t npt,
                     const double* params, int32_t npv, const int32_t* supersampling,
                     const double* exptime, int32_t* pv_status, void* workspace,
                     size_t workspace_bytes, void* stream);
rr_status rr_evaluate_prepared(rr_ctx* ctx, const double* times, const int32_t* pb_index, int32_t npt,
                               const double* params, int32_t npv, const int32_t* supersampling,
                               const double* exptime, void* flux, int32_t* pv_status,
                               const void* workspace, size_t workspace_bytes, void* stream);
rr_status rr_evaluate_grad_prepared(rr_ctx* ctx, const double* times, const int32_t* pb_index,
                                    int32_t npt, const double* params, int32_t npv,
                                    const int32_t* supersampling, const double* exptime,
                                    const void* grad_flux, double* grad_params, int32_t* pv_status,
                                    const void* workspace, size_t workspace_bytes, void* stream);

/* The light curves and the adjoint of a prepared batch for a cotangent known
 * in advance (Eq. 5 and the vector-Jacobian product of rr_evaluate_grad):
 * rr_evaluate_prepared and rr_evaluate_grad_prepared in one call, the adjoint
 * on a second stream of the context that forks from `stream` and joins it
 * again, so that the adjoint (latency-bound) runs beside the forward kernel
 * (an output stream).  Arguments as the two calls; flux and grad_params both
 * written; results bitwise those of the two calls.  The paper has no
 * counterpart.  The context's second stream is created on first use and
 * freed by rr_destroy; like every entry point, calls on one context must not
 * overlap in time.  Errors: as the two calls, plus RR_ECUDA for the stream
 * or its events. */
rr_status rr_evaluate_both_prepared(rr_ctx* ctx, const double* times, const int32_t* pb_index,
                                    int32_t npt, const double* params, int32_t npv,
                                    const int32_t* supersampling, const double* exptime,
                                    const void* grad_flux, void* flux, double* grad_params,
                                    int32_t* pv_status, const void* workspace, size_t workspace_bytes,
                                    void* stream);

/* Evaluate host-resident batches: host arrays in, host arrays out.  Light
 * curves (Eq. 5 with the supersampling of Sect. 4.1) and, when grad_flux is
 * given, the adjoint of rr_evaluate_grad, for data that live in host memory.
 * The paper has no counterpart (its models take and return host arrays, with
 * the GPU model copying them whole).
 *   In place: when every host array is page-locked memory mapped for the
 *   device (cudaHostAlloc, cudaHostRegister on a unified address space;
 *   both ends of each array are checked with cudaPointerGetAttributes), the
 *   kernels read the inputs and write the results where they are, over the
 *   host-device link, with no staging copies (the adjoint reads only the
 *   cotangent rows of the samples that may transit); chunk_pvs is unused.
 *   Staged: otherwise the batch is cut into chunks of chunk_pvs parameter
 *   vectors (0: npv / 8, at least 512); the copies of chunk c to the device,
 *   the kernels of chunk c-1 and the copies of chunk c-2 back to the host
 *   run on three streams of the context, so they overlap.
 *   times, pb_index, params, supersampling, exptime   host, as rr_evaluate
 *   grad_flux    host, [npv][npt] float (MIXED) / double (FP64), or NULL
 *                (no adjoint; grad_params is then not written)
 *   flux         host, [npv][npt] float (MIXED) / double (FP64), written
 *   grad_params  host, double[npv][nparam], written when grad_flux != NULL
 *   pv_status    host, int32[npv], or NULL
 * Host arrays should be page-locked (cudaHostAlloc / cudaHostRegister):
 * copies from pageable memory are staged by the driver and do not overlap.
 * The call is synchronous: it returns when every result is in host memory.
 * The context keeps one device buffer for the chunks or the in-place
 * workspace (grown when a call
 * needs more, freed by rr_destroy) and three streams; calls on one context
 * must not overlap in time (as for every entry point).  Results are bitwise
 * those of rr_evaluate / rr_evaluate_grad on the whole batch.
 * Errors: as rr_evaluate, plus RR_ECUDA for a failed copy or allocation and
 * RR_ETIMEOUT as reported by rr_sync_status. */
rr_status rr_evaluate_host(rr_ctx* ctx, const double* times, const int32_t* pb_index, int32_t npt,
                           const double* params, int32_t npv, const int32_t* supersampling,
                           const double* exptime, const void* grad_flux, void* flux, double* grad_params,
                           int32_t* pv_status, int32_t chunk_pvs);

/* One request from host buffers, asynchronous (serving: many requests in
 * flight on different streams).  Enqueues on `stream` the evaluation (with
 * one shared set-up and the adjoint when grad_flux != NULL) and returns once
 * everything is enqueued.  In place, as rr_evaluate_host, when every host
 * buffer is mapped page-locked memory (the kernels read and write them over
 * the host-device link; scratch holds the workspace only); otherwise staged:
 * copies of the host inputs into `scratch`, the kernels, and copies of
 * flux, pv_status and grad_params back to host memory.
 * The paper has no counterpart.  Arguments as rr_evaluate_host, plus
 *   scratch      device, >= rr_request_bytes(ctx, npv, npt, with_grad)
 *                bytes (in place, the workspace rr_workspace_bytes rounded
 *                up to 256 bytes suffices), 256-byte aligned, owned by the
 *                caller and not to be reused until the stream has passed
 *                this request
 * Host buffers must be page-locked for the copies to be asynchronous, and
 * must stay untouched until the stream has passed the request (an event
 * recorded after the call tells when).  Results are bitwise those of
 * rr_evaluate / rr_evaluate_grad.  Errors: as rr_evaluate, plus RR_ECUDA
 * for a failed copy. */
size_t rr_request_bytes(const rr_ctx* ctx, int32_t npv, int32_t npt, int32_t with_grad);
rr_status rr_enqueue_host(rr_ctx* ctx, const double* times, const int32_t* pb_index, int32_t npt,
                          const double* params, int32_t npv, const int32_t* supersampling,
                          const double* exptime, const void* grad_flux, void* flux, double* grad_params,
                          int32_t* pv_status, void* scratch, size_t scratch_bytes, void* stream);

/* Continuous-batching server (no counterpart in the paper): a worker thread
 * in the library admits queued requests in arrival order whenever one of its
 * `slots` streams is free and the request's device bytes (its workspace,
 * since a served request runs in place) fit in `mem_budget`; each admitted
 * request is enqueued with rr_enqueue_host on its own stream, with device
 * memory from a stream-ordered pool of the server; completion is detected
 * by polling events.  Work of
 * requests admitted at different times overlaps on the device, and a
 * request's results are those it would have alone.
 *   - While a context is used by a server, no other thread may call the
 *     library with that context.
 *   - Host buffers: page-locked and mapped for the device (cudaHostAlloc,
 *     cudaHostRegister), untouched by the caller until the request is
 *     reported finished by rr_server_poll.
 *   - rr_server_submit copies supersampling / exptime and returns the
 *     request id (>= 0), or a negative rr_status: -RR_EINVAL (arguments),
 *     -RR_EPAGEABLE (a host buffer, checked at both ends, is not page-locked
 *     memory mapped for the device), -RR_ENOMEM (larger than the budget),
 *     -RR_ESTATE (server stopping).
 *   - rr_server_submit_at is rr_server_submit with a release time: the
 *     request arrives at release_ns (rr_server_now_ns clock; 0 = now) and is
 *     not admitted before it.  Admission stays in submission order, so a
 *     caller gives non-decreasing release times.  A release time already past
 *     counts as the arrival all the same (an open-loop client that submits
 *     late has its lateness counted in the latency).
 *   - rr_server_now_ns: the library's steady clock (ns), the clock of every
 *     server time.
 *   - rr_server_poll hands over up to `max` finished requests (waiting up to
 *     timeout_us for the first): ids, their rr_status, and per request three
 *     steady-clock times in ns (arrival, admitted, finished); returns the
 *     count, or a negative rr_status.
 *   - rr_server_destroy finishes every queued request first. */
typedef struct rr_server rr_server;
rr_status rr_server_create(int32_t device, int32_t slots, size_t mem_budget, rr_server** out);
rr_status rr_server_destroy(rr_server* server);
int64_t rr_server_submit(rr_server* server, rr_ctx* fit, const double* times, const int32_t* pb_index,
                         int32_t npt, const double* params, int32_t npv, const int32_t* supersampling,
                         const double* exptime, const void* grad_flux, void* flux, double* grad_params,
                         int32_t* pv_status);
int64_t rr_server_submit_at(rr_server* server, rr_ctx* fit, const double* times, const int32_t* pb_index,
                            int32_t npt, const double* params, int32_t npv, const int32_t* supersampling,
                            const double* exptime, const void* grad_flux, void* flux, double* grad_params,
                            int32_t* pv_status, int64_t release_ns);
int64_t rr_server_now_ns(void);
int32_t rr_server_poll(rr_server* server, int64_t* ids, int32_t* status, int64_t* times_ns, int32_t max,
                       int32_t timeout_us);
/* Requests submitted and not yet handed over by rr_server_poll, minus those finished. */
int32_t rr_server_pending(rr_server* server);

/* Copy a set-up table to host memory (for inspection and tests); returns the
 * element count of the table, or -1 on error.  `out` may be NULL to query
 * the size; otherwise it receives min(count, capacity) doubles.
 *   RR_TABLE_ZE (nz+1), RR_TABLE_ZM (nz), RR_TABLE_MU (nz)
 *   RR_TABLE_WEIGHTS (nk*ng*nz), RR_TABLE_BASIS (nbasis*nz) profiles at zm,
 *   RR_TABLE_ISTAR (nbasis), RR_TABLE_PROJ (nbasis*nk*ng) = w . basis
 * Tables other than the grid need rr_build_weights first; the direct model
 * has no RR_TABLE_WEIGHTS or RR_TABLE_PROJ (-1, RR_ESTATE).  Synchronous. */
#define RR_TABLE_ZE 0
#define RR_TABLE_ZM 1
#define RR_TABLE_MU 2
#define RR_TABLE_WEIGHTS 3
#define RR_TABLE_BASIS 4
#define RR_TABLE_ISTAR 5
#define RR_TABLE_PROJ 6
int64_t rr_read_table(rr_ctx* ctx, int32_t which, double* out, int64_t capacity);

/* Exact flux (Sect. 2, Eq. 1 in radial form; no radial grid, no weights): for
 * planet-star distances z[i] and radius ratios k[i] (device, double[n]),
 *   out[i] = 1 - (1 / I_star) int_0^1 I(mu(r)) 2 r theta_i(r) dr  (device, double[n]),
 * theta the half-angle of the radius-r circle inside the planet (pi where the
 * planet covers the whole circle).  The law is the context's, with the
 * coefficients ldc (host, nldc values of one passband; Kipping q1, q2 for
 * RR_LD_QUADRATIC_TRI; ignored for a table) and passband pb's profile and
 * I_star.  FP64 Gauss-Legendre quadrature, 96 nodes per piece (the wholly
 * covered circles and the lens; 512 for a table), each piece mapped by
 * r = a + (b - a)(1 - cos phi) / 2 so that the square-root behaviour at the
 * contacts and at the limb is absorbed.  Accuracy: FP64 round-off for the
 * uniform, linear, quadratic and general laws; ~1e-10 for the nonlinear,
 * logarithmic and exponential laws (their mu^(1/2), mu ln mu, 1/(1 - e^mu)
 * terms stay non-smooth at the limb); ~1e-8 for a table (a kink at every
 * table node).  The reference of rr_choose_grid.
 * Enqueued on `stream`; needs rr_build_weights.  Errors: RR_EINVAL,
 * RR_ESTATE, RR_ECUDA. */
rr_status rr_exact_flux(rr_ctx* ctx, const double* z, const double* k, int32_t n, const double* ldc,
                        int32_t pb, double* out, void* stream);

/* Automatic grid resolution (Sect. 3.1.1 and 3.3: the resolutions and z_cut
 * chosen for a limb-darkening law and an error threshold).  Searches the
 * radial grid and the g grid for the direct model (FP64) whose flux stays
 * within `target` (absolute) of rr_exact_flux for every radius ratio k[0..nk)
 * (0 < k < 1, nk <= 64) at 400 planet positions each (g = 0 and a golden-ratio
 * sequence over [0, 0.999)), with the law cfg->ld_model (cfg->ncoef), the
 * coefficients ldc (host) or, for RR_LD_TABULATED, the profile (mu_tab,
 * I_tab, ntab).  Ladders: nzin, nzlimb in {4, 6, 8, 12, ..., 2048}, ng in
 * {10, 15, 20, 30, ..., 3840}, z_cut in {0.5, 0.6, 0.7, 0.8, 0.9}.  Greedy:
 * from (0.7, 8, 8, 20) take the step with the largest error reduction per
 * unit of added cost (nz x ng) until the target is met, then coarsen each
 * dimension while it stays met.  Writes zcut, nzin, nzlimb, ng of *cfg (the
 * other fields are read: ld_model, ncoef, device) and the achieved largest
 * error to *max_err.  Synchronous; creates and destroys its own contexts.
 * Errors: RR_EINVAL, RR_ECUDA, RR_EDOMAIN (target not reached on the ladders;
 * *cfg and *max_err hold the best grid found). */
rr_status rr_choose_grid(rr_config* cfg, const double* k, int32_t nk, const double* ldc, const double* mu_tab,
                         const double* I_tab, int32_t ntab, double target, double* max_err);

/* Synchronise `stream` and report whether any kernel of this context gave up
 * a bounded device-side wait since the last check (RR_ETIMEOUT; the affected
 * outputs are incomplete).  Resets the indicator.  Errors: RR_ECUDA. */
rr_status rr_sync_status(rr_ctx* ctx, void* stream);

/* Failure-detection self-test (no fault, trap or hang): enqueue on `stream` a
 * one-CTA kernel whose bounded device-side wait runs out on purpose --
 * which = 0: an mbarrier phase whose expected bytes never arrive (the wait of
 * the shared-memory staging copies, about one second); which = 1: a work-queue
 * slot that no producer publishes (the queue's claim wait, tens of ms).  The
 * kernel records the expiry in the context's error word and returns, so the
 * next rr_sync_status reports RR_ETIMEOUT and the context stays usable.
 * Errors: RR_EINVAL (which), RR_ECUDA. */
rr_status rr_selftest_wait(rr_ctx* ctx, int32_t which, void* stream);

/* Description of the last error on `ctx` (or of the last rr_create failure
 * when ctx is NULL).  Valid until the next call on the same context. */
const char* rr_last_error(const rr_ctx* ctx);

/* Count of kernel launches this context has issued since creation. */
int64_t rr_launch_count(const rr_ctx* ctx);

/* Kernel kinds for per-kernel timing. */
#define RR_KERNEL_LD_BASIS 0
#define RR_KERNEL_WEIGHTS 1
#define RR_KERNEL_PV_SETUP 2
#define RR_KERNEL_FLUX 3
#define RR_KERNEL_GRAD 4
#define RR_KERNEL_GRAD_REDUCE 5
#define RR_KERNEL_POINTS 6    /* several passbands; with one, the per-time preparation is part of PV_SETUP */
#define RR_KERNEL_DIRECT 7    /* the direct model's per-call weight projections */
#define RR_KERNEL_KINDS 8

/* Per-kernel timing (measurement aid).  While enabled, every kernel launch
 * of this context is bracketed by two CUDA events recorded on the launching
 * stream.  rr_profile_read waits for the recorded events, adds their elapsed
 * times to per-kind totals, and returns the total milliseconds and launch
 * count of `kind` (optionally resetting all totals).  Errors: RR_EINVAL. */
rr_status rr_profile(rr_ctx* ctx, int32_t enable);
rr_status rr_profile_read(rr_ctx* ctx, int32_t kind, double* total_ms, int64_t* count, int32_t reset);

/* Sample counts (measurement aid; the paper has no counterpart): while
 * enabled, the mixed-precision flux and adjoint kernels run in a counting form
 * (same results) that adds the work of every sample into per-kind counters:
 *   RR_COUNT_TIMES     candidate times (times whose exposure can overlap a
 *                      transit window): the float-float phase
 *   RR_COUNT_SAMPLES   their exposure sub-samples: offset and window test
 *   RR_COUNT_ORBIT     of those, samples inside the window: the orbit
 *   RR_COUNT_CIRCULAR  of the orbits, circular ones (no Kepler solve)
 *   RR_COUNT_NEWTON    Newton iterations of the FP32 Kepler solves
 *   RR_COUNT_TRANSIT   samples in transit: covered area and profile lookup
 *                      (the adjoint: with every partial derivative)
 *   RR_COUNT_LENS      of those, samples on the stellar limb (ingress and
 *                      egress: the lens area with its square root and two
 *                      arctangents; the others have the planet's whole area)
 *   RR_COUNT_REFINED   adjoint samples recomputed in float-float near a
 *                      contact point or a g-node
 * rr_count_read copies the counters of kernel kind RR_KERNEL_FLUX or
 * RR_KERNEL_GRAD into counts[RR_COUNT_KINDS] (synchronising the device) and
 * optionally resets all of them.  The counting form is slower: time the
 * kernels with counting off.  Errors: RR_EINVAL, RR_ENOMEM, RR_ECUDA. */
#define RR_COUNT_TIMES 0
#define RR_COUNT_SAMPLES 1
#define RR_COUNT_ORBIT 2
#define RR_COUNT_CIRCULAR 3
#define RR_COUNT_NEWTON 4
#define RR_COUNT_TRANSIT 5
#define RR_COUNT_REFINED 6
#define RR_COUNT_LENS 7
#define RR_COUNT_KINDS 8
rr_status rr_count_samples(rr_ctx* ctx, int32_t enable);
rr_status rr_count_read(rr_ctx* ctx, int32_t kind, int64_t* counts, int32_t reset);

/* How the last rr_evaluate_host / rr_enqueue_host call on the context ran:
 * RR_HOST_IN_PLACE (the kernels read and wrote the mapped page-locked host
 * buffers), RR_HOST_STAGED (copies through device buffers), or 0 (no such
 * call yet, or ctx NULL).  Introspection only; no counterpart in the paper. */
#define RR_HOST_IN_PLACE 1
#define RR_HOST_STAGED 2
int32_t rr_host_path(const rr_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* RR_H */

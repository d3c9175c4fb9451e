/*
 * musr.h -- C ABI of libmusr, a GB300 (sm_103a) implementation of the muSR
 * chi^2 / Poisson -2lnL cost and its analytic gradient (arXiv 1509.07685,
 * Section 4 "Parameter Fitting with Minuit2").
 *
 * What the library evaluates (Section 4.1):
 *   Eq. positron_histo   N_j(t) = N0_j exp(-t/tau_mu) [1 + A_j(p, t)] + Nbkg_j
 *   Eq. chisq            chi^2  = sum_j sum_n (d - N)^2 / max(d, 1)
 *   Eq. log-likelihood   -2lnL  = 2 sum_j sum_n [(N - d) + d ln(d/N)]  (d > 0)
 *                                                [ N - d ]            (d <= 0)
 *   Eq. asymmetry        A(t) = sum of terms, each a product of primitives
 *                        AMP(a) = a, EXP(lambda) = exp(-lambda t),
 *                        GAUSS(sigma) = exp(-(sigma t)^2 / 2),
 *                        KT(Delta) = 1/3 + 2/3 (1 - Delta^2 t^2) exp(-Delta^2 t^2 / 2),
 *                        TFCOS(nu, phi) = cos(2 pi (nu t + phi / 360)).
 * Units: t in microseconds, rates in 1/us, nu in MHz, phi in degrees,
 * tau_mu = 2.197019 us.  The time of bin n of histogram j is
 * t_n = (n - t0_j) * (bin_width_ns / 1000.0); a bin is in the fit when
 * fit_lo <= t_n <= fit_hi (closed range).  Local parameter slot 0 of every
 * histogram is N0, slot 1 is Nbkg; terms reference any slot.
 *
 * As in the paper's offload (Section 4, "The DKS Implementation"), the
 * histograms cross to the device once; per evaluation only the parameter
 * vector goes in and (1 + P) doubles (value and gradient) come back.
 *
 * Conventions for every entry point:
 *   - returns a musr_status (0 on success, negative on error); nothing is
 *     thrown across the ABI; musr_last_error() describes the last failure;
 *   - host arrays passed in are copied before the call returns, unless the
 *     entry point says it borrows them; host output arrays are owned by the
 *     caller;
 *   - one musr_ctx is not thread-safe: use one per thread.
 */
#ifndef MUSR_H_
#define MUSR_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MUSR_OK = 0,
  MUSR_EINVAL = -1,     /* invalid argument or inconsistent configuration */
  MUSR_ENOMEM = -2,     /* host or device allocation failed, or HBM budget exceeded */
  MUSR_ECUDA = -3,      /* a CUDA runtime call failed (see musr_last_error) */
  MUSR_ENONFINITE = -4, /* the cost is not finite: -2lnL with N <= 0 in a bin with d > 0, or a
                           parameter that is not finite */
  MUSR_ETIMEOUT = -5,   /* a bounded wait on the host ran out (musr_sync, musr_server_wait) */
  MUSR_ESTATE = -6,     /* call order violated (e.g. eval before upload) */
  MUSR_EAGAIN = -7,     /* result not ready yet (serving poll) */
  MUSR_ECANCELED = -8   /* a served fit was canceled (musr_server_cancel) */
} musr_status;

enum { MUSR_DTYPE_INT32 = 0, MUSR_DTYPE_FP32 = 1, MUSR_DTYPE_FP64 = 2 };
enum { MUSR_CHI2 = 0, MUSR_MLE = 1 };
/* MUSR_FP64: every per-bin operation in FP64 (the plain path).
 * MUSR_SPLIT: per-bin theory, residuals and gradient terms in FP32; FP64 for
 * the phase range reduction of 2 pi (nu t + phi/360) and for every
 * accumulation above the thread (block, grid, final sum).  Theories whose
 * terms factor into shared time functions with per-histogram coefficients use
 * that basis form; others (a stretched exponential, a Bessel precession, two
 * cosines in one term) evaluate the term list per bin in FP32. */
enum { MUSR_FP64 = 0, MUSR_SPLIT = 1 };
enum {
  MUSR_PRIM_AMP = 1,
  MUSR_PRIM_EXP = 2,
  MUSR_PRIM_GAUSS = 3,
  MUSR_PRIM_KT = 4,
  MUSR_PRIM_TFCOS = 5, /* slot[0] = nu (MHz), slot[1] = phi (degrees) */
  MUSR_PRIM_LKT = 6,   /* static Lorentzian Kubo-Toyabe 1/3 + 2/3 (1 - a t) exp(-a t); slot[0] = a (1/us) */
  MUSR_PRIM_STREXP = 7, /* stretched exponential exp(-(|lambda| t)^beta) for t > 0, 1 for t <= 0;
                           slot[0] = lambda (1/us), slot[1] = beta */
  MUSR_PRIM_BESSEL = 8, /* J0(2 pi (nu t + phi / 360)), Bessel precession (incommensurate order);
                           slot[0] = nu (MHz), slot[1] = phi (degrees) */
  MUSR_PRIM_DKT = 9     /* dynamic Gaussian Kubo-Toyabe relaxation of the strong-collision model
                           (fields of width Delta drawn anew at rate nu): the solution G of
                           G(t) = f(t) + nu int_0^t f(s) G(t - s) ds, f = KT(Delta, t) exp(-nu t),
                           1 for t <= 0; slot[0] = Delta (1/us), slot[1] = nu (1/us).  Evaluated
                           from a table solved on the device per evaluation (relative accuracy
                           of order 1e-6); at most 8 distinct (Delta, nu) pairs per context;
                           not in serving requests or musr_eval_noalloc */
};

#define MUSR_MAX_PRIMS 4
#define MUSR_MAX_TERMS 4
#define MUSR_MAX_SLOTS 32
#define MUSR_MAX_PARAMS 4096

/* One term of A(t): the product of nprim primitives (Eq. asymmetry,
 * generalised).  slot[m][0] (and slot[m][1] for the two-slot primitives TFCOS, STREXP,
 * BESSEL, DKT) are local slots. */
typedef struct musr_term {
  int32_t nprim;
  int32_t kind[MUSR_MAX_PRIMS];
  int32_t slot[MUSR_MAX_PRIMS][2];
} musr_term;

typedef struct musr_ctx musr_ctx;

/* Creates a context on CUDA device `device`.  hbm_budget_bytes caps the
 * device memory the context may allocate (0: no cap).  cuda_stream is a
 * cudaStream_t to run on (e.g. torch.cuda.current_stream().cuda_stream; the
 * legacy default stream is passed as cudaStreamLegacy, (void*)1), or NULL for
 * a stream the context creates.  The context owns all memory it
 * allocates; *out is NULL on failure.  (Section 2.1: memory handling and
 * streams of the DKS communication layer.) */
int musr_ctx_create(musr_ctx** out, int device, size_t hbm_budget_bytes, void* cuda_stream);

/* Frees everything the context owns.  NULL is ignored. */
void musr_ctx_destroy(musr_ctx* ctx);

/* Text of the last error on this context ("" if none).  ctx NULL: the last error
 * of musr_ctx_create or musr_eval_noalloc on the calling thread.  The pointer stays
 * valid until the next call. */
const char* musr_last_error(const musr_ctx* ctx);

/* Copies nhist histograms of nbins bins (host, row-major [nhist][nbins]) to
 * the device, once (Section 4, "The DKS Implementation": measurement data
 * go to the device at the beginning).  dtype is MUSR_DTYPE_INT32 (stored as
 * FP32; |count| must be < 2^24 so the copy is exact), MUSR_DTYPE_FP32 or
 * MUSR_DTYPE_FP64 (stored as FP64).  t0[nhist] is the time-zero bin of each
 * histogram (may be fractional), bin_width_ns > 0, fit_range_us = {lo, hi}.
 * Replaces any previous histograms; theory and map must be (re)set after.
 * The rows are copied as they are and checked on the device (a count that is
 * not finite, or an INT32 count beyond 2^24, gives MUSR_EINVAL and no
 * histograms).  Synchronous: the caller may reuse `counts` when it returns. */
int musr_upload_histograms(musr_ctx* ctx, const void* counts, int dtype, int nhist, int64_t nbins,
                           const double* t0, double bin_width_ns, const double fit_range_us[2]);

/* Uploads asymmetry data instead of histograms (the asymmetry A(t) of
 * Eq. asymmetry measured directly): npairs forward / backward histogram pairs,
 * forward and backward host arrays [npairs][nbins] in `dtype` (as for
 * musr_upload_histograms), the relative efficiency alpha[npairs] > 0 and the
 * constant backgrounds bkg_forward[npairs], bkg_backward[npairs] (counts per
 * bin) of each pair.  On the device, with f = F - bkg_F and b = B - bkg_B,
 *     a = (f - alpha b) / (f + alpha b),
 *     w = 1 / sigma_a^2,  sigma_a^2 = 4 alpha^2 (b^2 max(F,1) + f^2 max(B,1))
 *                                     / (f + alpha b)^4
 * (first-order propagation of the Poisson errors of F and B), w = 0 where
 * f + alpha b <= 0; a and w are kept in FP64.  The context then evaluates the
 * asymmetry model T(t) = N0 A(t) + Nbkg (no decay envelope: local slot 0 is a
 * scale, usually mapped to the constant 1, slot 1 a baseline) with the cost
 * chi^2 = sum w (a - T)^2: mode MUSR_CHI2 only (MUSR_MLE gives MUSR_EINVAL);
 * Gauss-Newton products at MUSR_FP64 precision only.  t0, bin_width_ns and
 * fit_range_us as for musr_upload_histograms; counts are checked the same way.
 * Replaces any previous data; theory and map must be (re)set after.
 * Synchronous: the caller may reuse its arrays when it returns. */
int musr_upload_asymmetry(musr_ctx* ctx, const void* forward, const void* backward, int dtype, int npairs,
                          int64_t nbins, const double* t0, double bin_width_ns, const double fit_range_us[2],
                          const double* alpha, const double* bkg_forward, const double* bkg_backward);

/* As musr_upload_histograms, but BORROWS device memory the caller owns
 * (e.g. a torch tensor): d_counts points to [nhist][row_stride] FP32 or FP64
 * values on the context's device, 16-byte aligned, row_stride a multiple of 4
 * elements and >= nbins.  The memory must stay valid and unchanged until the
 * histograms are replaced or the context is destroyed. */
int musr_upload_histograms_device(musr_ctx* ctx, const void* d_counts, int dtype, int nhist,
                                  int64_t nbins, int64_t row_stride, const double* t0,
                                  double bin_width_ns, const double fit_range_us[2]);

/* Sets A(t) as nterms (<= MUSR_MAX_TERMS) terms (Section 4.1: Eq. asymmetry writes
 * A(t) as an amplitude times relaxation and precession factors; the paper's fits take
 * any "user defined function" of the parameters in its place, here any sum of up to
 * four products of up to four of the primitives above).  terms is a host array, copied.
 * Every slot referenced must be < the nslots given to musr_set_map.  MUSR_EINVAL for an
 * unknown primitive, a slot out of range or more than four terms or primitives; the
 * map must be set again after a new theory. */
int musr_set_theory(musr_ctx* ctx, const musr_term* terms, int nterms);

/* Sets the per-histogram parameter map (Section 4.1: the parameter set
 * P_j = {N0_j, Nbkg_j, p_j} of each detector drawn from one global vector).
 * map is [nhist][nslots] int32: entry m >= 0 takes global parameter m
 * (< nparams); m < 0 takes consts[-1 - m] (< nconsts).  Requires histograms
 * and theory.  nslots <= MUSR_MAX_SLOTS, nparams <= MUSR_MAX_PARAMS. */
int musr_set_map(musr_ctx* ctx, const int32_t* map, int nslots, int nparams, const double* consts,
                 int nconsts);

/* Evaluates the cost (mode MUSR_CHI2: Eq. chisq; MUSR_MLE: Eq. log-likelihood)
 * at params[nparams] (host) in the given precision.  *out_value receives the
 * cost; out_grad[nparams] (host, may be NULL for value only) the analytic
 * gradient.  Synchronous on the context's stream.  Returns MUSR_ENONFINITE
 * (value +inf, grad zeros) when the likelihood is undefined. */
int musr_eval(musr_ctx* ctx, const double* params, int nparams, int mode, int precision,
              double* out_value, double* out_grad);

/* Gauss-Newton products for parameter error estimates (Section 4.1: the
 * minimiser's parameter errors come from the curvature of the cost).  With J the
 * parameter gradient of every bin's expected count N (Eq. positron_histo), the
 * Gauss-Newton matrix is H = sum over bins of (d^2 cost / dN^2) J J^T, where
 * d^2/dN^2 is 2/max(d,1) for Eq. chisq and 2d/N^2 for Eq. log-likelihood (the
 * Hessian of the cost without the term in d cost/dN, which vanishes where the
 * model fits).  For each of ndir directions v (host dirs[ndir][nparams]) at host
 * params[nparams]: out[ndir][1 + nparams] (host) receives v^T H v and H v.
 * One launch for all directions; synchronous on the context's stream.
 * Returns MUSR_ENONFINITE (row zeros after an infinite first entry) where the
 * likelihood is undefined.  At MUSR_SPLIT precision only for theories with a
 * basis form and histogram data (else MUSR_EINVAL: use MUSR_FP64). */
int musr_gn_product(musr_ctx* ctx, const double* params, int nparams, const double* dirs, int ndir, int mode,
                    int precision, double* out);

/* The whole Gauss-Newton matrix at params: out[nparams][nparams] (host),
 * symmetrised (H + H^T)/2 from the products with every unit vector (one launch).
 * The parameter errors of a fit at its optimum are sqrt(2 (H^-1)_ii) (both costs
 * are -2 ln L scaled, so a change of 1 in the cost is one standard deviation). */
int musr_gauss_newton(musr_ctx* ctx, const double* params, int nparams, int mode, int precision, double* out);

/* nvec evaluations in one launch (e.g. trial points of a line search, or
 * the random parameter vectors of a scan): params is host [nvec][nparams],
 * out_values host [nvec], out_grads host [nvec][nparams] or NULL.  Returns
 * MUSR_ENONFINITE if any vector's likelihood is undefined (its value is +inf). */
int musr_eval_batch(musr_ctx* ctx, const double* params, int nvec, int nparams, int mode,
                    int precision, double* out_values, double* out_grads);

/* Device-resident variant for callers that keep everything in HBM (torch
 * tensors): d_params is device [nvec][nparams] FP64, d_out device
 * [nvec][1 + nparams] FP64 (value, then gradient; with_grad == 0 writes the
 * value only).  Asynchronous: enqueued on the context's stream, nothing is
 * copied or synchronised.  A +inf value marks an undefined likelihood. */
int musr_eval_device(musr_ctx* ctx, const double* d_params, int nvec, int mode, int precision,
                     int with_grad, double* d_out);

/* Waits (bounded by timeout_ms, <= 0: no bound) for the context's stream. */
int musr_sync(musr_ctx* ctx, int timeout_ms);

/* Number of (histogram, bin) pairs inside the fit range. */
int musr_bins_in_fit(musr_ctx* ctx, int64_t* out);

/* The error word of the kernels' index checks (no counterpart in the paper).  The library
 * built with MUSR_DEBUG_CHECKS (paper_1509_07685_gb300/build.py, debug=True: libmusr_debug.so)
 * tests every computed index against its bounds on the device; a check that fails ORs its
 * bit into the context's word and skips the access, nothing traps.  Bits: 1 a count or
 * weight beyond its row, 2 a histogram index, 4 a chunk or item index, 8 a partial row,
 * 16 a parameter-map entry, 32 a dynamic Kubo-Toyabe table, 64 a finalize column, 128 a
 * job index.  Waits for the context's stream and returns the word accumulated since the
 * context's first evaluation (0: no check failed).  The release build returns MUSR_ESTATE
 * and 0. */
int musr_debug_word(musr_ctx* ctx, uint32_t* out);

/* Number of kernel launches one musr_eval/musr_eval_batch/musr_eval_device
 * call makes (for launch accounting). */
int musr_launches_per_eval(musr_ctx* ctx, int* out);

/* ---------------------------------------------------------------------------
 * Fitting (Section 4: the minimiser runs on the host, each trial point is one
 * cost evaluation on the device; a project-written BFGS stands in for migrad).
 * ------------------------------------------------------------------------- */

/* Outcome of one fit.  status: 0 converged, 1 cost non-finite at the start,
 * 2 iteration limit, 3 line search failed, < 0 a musr_status error. */
typedef struct musr_fit_result {
  int32_t status;
  int32_t iters;
  int32_t nfev;    /* cost evaluations (each a value and a gradient) */
  int32_t nparams;
  double f;        /* cost at the result */
  double edm;      /* estimated distance to the minimum, g.H^-1.g / 2 (cost units) */
  double t_submit; /* serving clock, seconds: submission, admission, completion */
  double t_admit;
  double t_done;   /* musr_fit: wall time of the fit */
} musr_fit_result;

/* Runs a BFGS fit of the context's problem from x0[nparams] (host) in the given
 * cost mode and precision; maxit <= 0 means 1000, gtol <= 0 means 1e-8.  Stops
 * when max|g| <= gtol max(1,|f|), when the estimated distance to the minimum is
 * below 1e-7 (FP64) or 1e-5 (SPLIT, whose FP32 gradient has a rounding floor),
 * or at maxit.  x_out[nparams] receives the result.  Synchronous. */
int musr_fit(musr_ctx* ctx, const double* x0, int mode, int precision, int maxit, double gtol,
             double* x_out, musr_fit_result* res);

/* ---------------------------------------------------------------------------
 * Serving: many fits at once (continuous batching).  A worker thread keeps
 * every admitted fit's histograms resident, evaluates the next trial point of
 * every active fit in one multi-fit launch per (precision, theory shape, cost)
 * group per step, and advances each fit's minimiser; fits that arrive while
 * others run are admitted at the next step boundary, as device memory within
 * the budget allows.  A fit's result does not depend on the other fits.
 * ------------------------------------------------------------------------- */

typedef struct musr_server musr_server;

/* One fit: the arguments of musr_upload_histograms, musr_set_theory and
 * musr_set_map, a start point, and the fit settings.  All arrays are host
 * memory, copied by musr_server_submit -- except the counts when flags holds
 * MUSR_REQ_BORROW_COUNTS: then the server reads them when it admits the fit,
 * and the caller keeps them valid and unchanged until the fit's result has
 * been taken (musr_server_poll / musr_server_wait) or the server destroyed. */
#define MUSR_REQ_BORROW_COUNTS 1
typedef struct musr_fit_request {
  const void* counts;
  int32_t dtype;
  int32_t nhist;
  int64_t nbins;
  const double* t0;
  double bin_width_ns;
  double fit_range_us[2];
  const musr_term* terms;
  int32_t nterms;
  int32_t nslots;
  const int32_t* map;
  int32_t nparams;
  int32_t nconsts;
  const double* consts;
  const double* x0;
  int32_t mode;
  int32_t precision;
  int32_t maxit; /* <= 0: 1000 */
  int32_t flags; /* 0 or MUSR_REQ_BORROW_COUNTS */
  double gtol;   /* <= 0: 1e-8 */
} musr_fit_request;

typedef struct musr_server_stats {
  int64_t submitted, completed, rejected, canceled;
  int64_t steps, launches, evals;
  int64_t active, queued;
  double bin_evals; /* (histogram, bin) pairs evaluated, summed over evaluations */
  double busy_s;    /* worker time inside steps */
  double clock_s;   /* serving clock now */
  uint64_t arena_bytes, arena_used;
  double minimizer_s; /* worker time in the fits' minimiser steps (trial points, updates) */
  double admit_s;     /* worker time admitting fits (contexts, uploads), overlapped with the device */
  double wait_s;      /* worker time waiting for the device */
  /* time configuring admitted fits, summed over the threads that did it: the context,
   * the histogram upload (enqueueing its copy and device check), theory + map +
   * planning, and the device tables and evaluation buffers with the wait for all of
   * the fit's setup work on the device */
  double cfg_create_s, cfg_upload_s, cfg_plan_s, cfg_buffers_s;
} musr_server_stats;

/* Starts a server on `device` with a device memory budget of hbm_budget_bytes
 * (one allocation, carved per fit) and at most max_active fits in flight. */
int musr_server_create(musr_server** out, int device, size_t hbm_budget_bytes, int max_active);

/* Stops the worker (running fits are abandoned) and frees everything. */
void musr_server_destroy(musr_server* s);

/* Queues a fit; *out_id identifies it.  Thread-safe.  A fit that can never run
 * (larger than the whole budget, bad arguments) ends
 * with a negative status instead of being queued forever. */
int musr_server_submit(musr_server* s, const musr_fit_request* req, int64_t* out_id);

/* MUSR_OK and the result (x_out[nparams], may be NULL) if fit `id` is done --
 * the result is then handed over and forgotten -- MUSR_EAGAIN if not yet. */
int musr_server_poll(musr_server* s, int64_t id, musr_fit_result* res, double* x_out);

/* As musr_server_poll, waiting at most timeout_ms (<= 0: without limit);
 * MUSR_ETIMEOUT if the fit is not done by then. */
int musr_server_wait(musr_server* s, int64_t id, int timeout_ms, musr_fit_result* res, double* x_out);

/* Asks fit `id` to stop.  A fit still queued ends at once without running; one being
 * admitted or running ends at its next step boundary, when none of its work is on the
 * device (its memory then goes back to the budget).  Either way its result, taken with
 * musr_server_poll / musr_server_wait as usual, has status MUSR_ECANCELED and the point it
 * had reached (x0 if it never ran).  Returns MUSR_OK when the fit was queued or running,
 * MUSR_ESTATE when it had finished already (its result stands), MUSR_EINVAL for an id
 * never issued or whose result was taken.  Thread-safe; it does not wait. */
int musr_server_cancel(musr_server* s, int64_t id);

/* Counters of the server.  completed counts fits that ran to an end of their own
 * (converged or stopped by the minimiser, or a device error); canceled the fits ended by
 * musr_server_cancel; rejected the fits refused at admission. */
int musr_server_stats_get(musr_server* s, musr_server_stats* out);

/* The paper has no counterpart to this entry point.
 *
 * One evaluation (value and, with with_grad != 0, gradient) that allocates no
 * memory, for callers that cannot allocate device memory: code inside a
 * framework whose memory pool owns the GPU and forbids cudaMalloc beside it,
 * plugins whose host reserves all HBM up front, or loops where the implicit
 * synchronisation of an allocation is not acceptable.  Such callers cannot
 * create a musr_ctx (a context allocates), so everything comes from them:
 * d_counts [nhist][row_stride] FP32 or FP64 on the current device (16-byte
 * aligned, row_stride a multiple of 4), d_params [nparams] FP64 on the device,
 * d_out [1 + nparams] FP64 on the device (value, then gradient); t0 [nhist], the
 * fit range, terms [nterms], map [nhist][nslots] and consts [nconsts] are host
 * arrays, read before the call returns.  Their meaning is that of
 * musr_upload_histograms, musr_set_theory and musr_set_map, and every theory
 * those accept runs here too (at MUSR_SPLIT, one without a basis form evaluates
 * its term list per bin), except one with the dynamic Kubo-Toyabe primitive
 * MUSR_PRIM_DKT, whose per-evaluation tables have no room here (MUSR_EINVAL).
 * The call is asynchronous on cuda_stream (NULL: the
 * legacy default stream).  d_out[0] is +inf where the likelihood is undefined or a
 * parameter is not finite (the call has returned MUSR_OK by then: read the value before
 * trusting the gradient).
 *
 * All scratch (work tables, partial sums, completion counters) lives in one
 * file-scope device array of MUSR_NOALLOC_SCRATCH_BYTES that every GPU which
 * loads the library holds until the process exits; with lazy module loading
 * the array is placed on a device at the first call there, so make that call
 * before a memory pool reserves the rest of the device.  Limits: nhist <= 64,
 * nparams <= 1024, nconsts <= 256, at most 8192 work items, and the scratch
 * size.  Every argument and limit check runs on the host before any CUDA call,
 * except the work-item count and the scratch size, which depend on the
 * device's SM count and are checked after the set-up below; every failure
 * returns MUSR_EINVAL (or MUSR_ECUDA) with its reason in musr_last_error(NULL)
 * on the calling thread, and enqueues nothing.  The first call on a device
 * looks up the array's device address (set-up).  The tables are staged from a
 * host buffer that each call overwrites, so a call on a stream that is
 * capturing returns MUSR_EINVAL.  Every call on a device uses the same array
 * and leaves its contents behind (the counters are cleared at the start of each
 * call): calls that overlap on the GPU race, so serialise them (one stream, or
 * an event between them). */
#define MUSR_NOALLOC_SCRATCH_BYTES (8u << 20)
int musr_eval_noalloc(const void* d_counts, int dtype, int nhist, int64_t nbins, int64_t row_stride,
                      const double* t0, double bin_width_ns, const double fit_range_us[2],
                      const musr_term* terms, int nterms, const int32_t* map, int nslots, int nparams,
                      const double* consts, int nconsts, const double* d_params, int mode,
                      int precision, int with_grad, double* d_out, void* cuda_stream);

/* The compute capability the library's kernels were compiled for, as the CUDA runtime
 * reports it for the code loaded on `device` (cudaFuncAttributes::binaryVersion: 103 for
 * sm_103a).  No counterpart in the paper: a build check.  MUSR_EINVAL for a bad device or a
 * NULL out; MUSR_ECUDA if the runtime cannot load the code for the device. */
int musr_binary_version(int device, int* out);

/* ---------------------------------------------------------------------------
 * The particle-mesh Poisson solve of Section 3 ("FFT Based Particle-Mesh
 * Solver"): the potential of an isolated charge density on an mx x my x mz
 * mesh with spacings hx, hy, hz,
 *     phi_{i,j,k} = hx hy hz sum rho_{i',j',k'} G_{i-i',j-j',k-k'},
 *     G_{a,b,c} = 1 / sqrt((a hx)^2 + (b hy)^2 + (c hz)^2)
 * (Eq. openbruteforceconv; G_{0,0,0}, where 1/r is singular, is 1/min(h)),
 * computed by Hockney's method (Eq. oneterm): the density zero-padded to the
 * doubled mesh, FP64 FFTs, the Hadamard product with the transform of G (real,
 * computed once per solver), the inverse FFT, the original block kept.
 * Arrays are [mx][my][mz] FP64, z fastest.
 * ------------------------------------------------------------------------- */

typedef struct musr_poisson musr_poisson;

/* Creates a solver for one mesh on CUDA device `device` (cuda_stream as for
 * musr_ctx_create; NULL: its own stream): allocates the doubled-mesh buffers
 * (about 48 mx my mz reals) and the FFT plans, and transforms G.  precision:
 * MUSR_FP64 (FP64 transforms) or MUSR_SPLIT (FP32 transforms between the FP64
 * density and potential; 2-norm relative error of phi below about
 * 10 log2(8 mx my mz) 2^-24, first-order FFT error bounds).  mx, my, mz >= 1
 * with 8 mx my mz < 2^31; spacings finite and > 0.  *out is NULL on failure
 * (MUSR_ENOMEM when the device has no room). */
int musr_poisson_create(musr_poisson** out, int device, int mx, int my, int mz, double hx, double hy, double hz,
                        int precision, void* cuda_stream);

/* Frees the solver.  NULL is ignored. */
void musr_poisson_destroy(musr_poisson* ps);

/* Text of the last error of the solver ("" if none); ps NULL: of the last
 * failed musr_poisson_create on this thread. */
const char* musr_poisson_last_error(const musr_poisson* ps);

/* phi [mx][my][mz] of rho [mx][my][mz], host arrays.  Synchronous: copies rho
 * in, solves, copies phi out. */
int musr_poisson_solve(musr_poisson* ps, const double* rho, double* phi);

/* The same on device arrays of the solver's device, enqueued on its stream
 * (returns before the solve ends; the arrays must stay valid until then). */
int musr_poisson_solve_device(musr_poisson* ps, const double* d_rho, double* d_phi);

#ifdef __cplusplus
}
#endif

#endif /* MUSR_H_ */

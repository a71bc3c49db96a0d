/*
 * nef.h -- C ABI of the GB300 (sm_103a) nonnegative einsum factorization engine.
 *
 * The engine fits  Yhat = einsum(model_str, Theta^(1), ..., Theta^(L))  to a
 * nonnegative tensor Y by the multiplicative update of NNEinFact:
 *   model family and model string ............ Sec. 2, Eq. 2.1-2.3
 *   objective with the floor eps ............. Sec. 3, Eq. 3.1
 *   update  Theta <- max(eps, Theta * g^{-1}(num/den)) ... Thm. 3.1, Eq. 3.4
 *   num/den as einsum(einstr_l, ...) ......... Eq. 3.5-3.8
 *   the sweep (Gauss-Seidel over factors) .... Algorithm 1
 *   (alpha,beta)-divergence, a, b and g ...... App. B
 *   missing data (mask) ...................... Sec. 6.5 (experimental design)
 *
 * Conventions shared by every entry point
 *   - Letters are lowercase a-z.  Letters on the right of "->" are observed
 *     (the modes of Y, in that order); letters that appear only on the left are
 *     latent (contracted), numbered in order of first appearance.
 *   - Y is row-major over the observed letters in right-hand-side order.
 *   - Factor l is row-major over the letters of the l-th term, in term order.
 *   - mask, when given, holds one byte per entry of Y (nonzero = observed).
 *   - Device pointers are CUDA global-memory pointers on the current device;
 *     the caller owns Y, mask and the factors.  Host pointers are marked.
 *   - Element type: double for NEF_FP64 plans, float otherwise (NEF_FP32 and
 *     NEF_BF16 keep FP32 data and FP32 master factors; NEF_BF16 feeds the
 *     tensor cores BF16 operands with FP32 accumulation).
 *   - Work is ordered on opt.stream (a cudaStream_t; NULL = legacy stream).
 *     nef_fit and nef_update return once the work is enqueued; nef_loss
 *     synchronises the stream.
 *   - No call throws or aborts: each returns a nef_status, and
 *     nef_last_error() gives a message for the last failure on this thread.
 *   - The plan owns a device workspace sized at nef_plan time; a plan may be
 *     used by one thread at a time.
 */
#ifndef NEF_H
#define NEF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nef_plan_s* nef_plan_t;

typedef enum {
    NEF_OK = 0,
    NEF_EINVAL = 1,        /* bad argument: null pointer, size, option or factor index   */
    NEF_EPARSE = 2,        /* malformed model string (Eq. 2.2 grammar)                    */
    NEF_EUNSUPPORTED = 3,  /* alpha == 0 with beta != 1 (no decomposition, App. B), or a  */
                           /* plan the requested precision cannot run                     */
    NEF_ENOMEM = 4,        /* device workspace allocation failed                          */
    NEF_ECUDA = 5,         /* a CUDA runtime or driver call failed                        */
    NEF_EDATA = 6,         /* Y holds a negative or non-finite entry (checked on request) */
    NEF_ETIMEOUT = 7       /* a bounded device-side wait gave up; the context is intact   */
} nef_status;

enum {
    NEF_FP32 = 0,  /* CUDA-core FP32 fused sweep (the plain FP32 path)                */
    NEF_BF16 = 1,  /* tcgen05 tensor cores: BF16 operands, FP32 TMEM accumulation     */
    NEF_FP64 = 2   /* CUDA-core FP64 fused sweep                                      */
};

/*
 * Loss families (nef_options.loss).  Each has the convex-concave structure of
 * Thm. 3.1, so Algorithm 1 applies with its own a(x, y), b(x, y) and g (App. B):
 *   NEF_LOSS_AB        (alpha,beta)-divergence D_{alpha,beta} (App. B, five cases);
 *                      the alpha, beta arguments of every call select it.
 *   NEF_LOSS_NEGBIN    negative binomial with dispersion phi = loss_par > 0 (one
 *                      value for every entry): D = (phi + x) log(phi + y) - x log y,
 *                      a = x / y, b = (phi + x) / (phi + y), g(l) = l (App. B,
 *                      negative binomial).
 *   NEF_LOSS_BINOMIAL  binomial on the odds y = p / (1 - p) with n = loss_par > 0
 *                      trials per entry (n = 1: Bernoulli): D = n log(1 + y) - x log y,
 *                      a = x / y, b = n / (1 + y), g(l) = l (App. B, Bernoulli and
 *                      binomial).  Per-entry trial counts are not supported.
 *   NEF_LOSS_JS        Jensen-Shannon: D = (x log x + y log y)/2 - m log m with
 *                      m = (x + y)/2, a = log((x + y) / (2 y)), b = 1, g = log, so the
 *                      update multiplies by exp(num / den) (App. B, Jensen-Shannon).
 * The constant terms of the log-likelihoods are dropped from D (0 log 0 = 0).
 * For the three likelihood families the alpha and beta arguments are ignored.
 */
enum {
    NEF_LOSS_AB = 0,
    NEF_LOSS_NEGBIN = 1,
    NEF_LOSS_BINOMIAL = 2,
    NEF_LOSS_JS = 3
};

typedef struct {
    int precision;      /* NEF_FP32, NEF_BF16 or NEF_FP64                                   */
    double eps;         /* floor of Eq. 3.1 (paper: "a very small eps > 0"); default 1e-10  */
    int check_data;     /* nonzero: nef_fit/nef_update first check Y >= 0 and finite        */
    int force_generic;  /* nonzero: use the unfused path (yhat, a, b materialised)          */
    int profile;        /* 1: time every fused-pass launch with CUDA events on the plan's   */
                        /* stream (nef_plan_profile); 2: also count wait and phase cycles   */
                        /* inside the tensor-core pass (nef_tc_trace; slows it down)        */
    void* stream;       /* cudaStream_t used by every call on the plan                      */
    double tol;         /* > 0: nef_fit stops after the first sweep k >= 2 whose preceding  */
                        /* relative loss decrease (L[k-2] - L[k-1]) / L[k-2] is below tol   */
                        /* (the training-loss stopping rule of App. B); 0 = exactly iters   */
    double* loss_trace; /* device, iters + 1 doubles, or NULL: loss_trace[k] = Eq. 3.1's    */
                        /* objective (sum over observed entries of D) after k sweeps;       */
                        /* entries past an early stop are left untouched                    */
    int eager;          /* nonzero: launch every kernel of every sweep directly; zero: from */
                        /* the third sweep on, replay a captured CUDA graph of one sweep    */
    int loss;           /* NEF_LOSS_AB (default), NEF_LOSS_NEGBIN, NEF_LOSS_BINOMIAL or     */
                        /* NEF_LOSS_JS: the loss every call on the plan fits and reports    */
    double loss_par;    /* phi for NEF_LOSS_NEGBIN, trials n for NEF_LOSS_BINOMIAL          */
    int64_t wait_cycles;/* limit, in SM clock cycles, of every bounded wait inside the      */
                        /* tensor-core pass; 0 = the default 4e9 (about 2 s).  A wait that  */
                        /* runs out stops its kernel cleanly and nef_check then reports     */
                        /* NEF_ETIMEOUT (the results of that call are invalid)              */
    int batch_tiles;    /* nef_fit_batched: 64-column tiles of Y per work item (one fused   */
                        /* pass of a row block over that many tiles); 0 = the default 64;   */
                        /* nef_fit_batched_tune picks one for a workload                    */
} nef_options;

/* Fill *opt with the defaults: NEF_FP32, eps = 1e-10, no data check, fused, no
 * profiling, stream NULL, tol 0, no loss trace, graph replay, NEF_LOSS_AB,
 * loss_par 0, default wait limit, default batched tiles per work item. */
void nef_default_options(nef_options* opt);

/*
 * nef_plan -- parse model_str (Eq. 2.2), check it, and build the per-factor
 * pass plans of Algorithm 1 (including swap(model_str, l) of Eq. 3.8).
 *   model_str : NUL-terminated, e.g. "ir,jr,kr->ijk" (host)
 *   shapes    : n_obs dimensions of Y in right-hand-side order (host)
 *   ranks     : n_lat latent dimensions in order of first appearance (host)
 *   opt       : options (host; NULL = defaults); copied into the plan
 *   out       : receives the plan handle (host)
 * Errors: NEF_EPARSE for a malformed string or a repeated letter within a
 * term or on the right; NEF_EINVAL for a count mismatch, a dimension < 1, an
 * unknown precision or loss, eps < 0, a loss_par outside its range (phi > 0,
 * n > 0, both finite) or wait_cycles < 0; NEF_ENOMEM / NEF_ECUDA from workspace
 * allocation.  On error *out is NULL.
 */
nef_status nef_plan(const char* model_str, const int64_t* shapes, int n_obs,
                    const int64_t* ranks, int n_lat, const nef_options* opt,
                    nef_plan_t* out);

/* Release the plan and its workspace (NULL is ignored). */
void nef_plan_destroy(nef_plan_t plan);

/*
 * nef_fit -- run `iters` sweeps of Algorithm 1: for l = 1..L in string order,
 * rebuild Yhat from the current factors, form num and den (Eq. 3.6-3.8) with
 * the masked weights a(Y,Yhat), b(Y,Yhat) of App. B, and apply Eq. 3.4.
 *   Y       : device, N elements (see conventions), not modified
 *   mask    : device, N bytes, or NULL (every entry observed)
 *   factors : host array of L device pointers, updated in place
 *   alpha, beta : the (alpha,beta)-divergence parameters of App. B
 *   iters   : number of sweeps (0 is a no-op)
 * The loss of the current factors is summed inside the first pass of every
 * sweep (its Yhat is already on chip) when opt.loss_trace or opt.tol asks for
 * it; one extra loss pass follows the last sweep.  With tol > 0 the stopping
 * rule runs on the device (as in nef_fit_ctl); nef_plan_sweeps reports how
 * many sweeps ran.
 * Errors: NEF_EUNSUPPORTED for alpha == 0 with beta != 1 (NEF_LOSS_AB plans);
 * NEF_EINVAL for a null pointer, iters < 0 or a non-finite alpha or beta;
 * NEF_EDATA if check_data found a bad Y entry (factors untouched); NEF_ECUDA
 * for a failed launch.
 */
nef_status nef_fit(nef_plan_t plan, const void* Y, const uint8_t* mask,
                   void* const* factors, double alpha, double beta, int iters);

/*
 * nef_fit_ex -- nef_fit with a per-call stopping tolerance and loss trace
 * (instead of the plan's opt.tol / opt.loss_trace).
 *   tol        : as nef_options.tol (0 = exactly iters sweeps)
 *   loss_trace : device, iters + 1 doubles, or NULL (as nef_options.loss_trace)
 *   sweeps     : host, receives the number of sweeps run, or NULL
 * Errors as nef_fit; NEF_EINVAL for tol < 0.
 */
nef_status nef_fit_ex(nef_plan_t plan, const void* Y, const uint8_t* mask, void* const* factors,
                      double alpha, double beta, int iters, double tol, double* loss_trace, int* sweeps);

/*
 * Stopping rules of App. B evaluated on the device, for nef_fit_ctl:
 *   tol          > 0: stop after the first sweep k >= 2 whose preceding relative
 *                training-loss decrease (L[k-2] - L[k-1]) / L[k-2] is below tol,
 *                L[k] being Eq. 3.1's objective after k sweeps (as nef_options.tol);
 *   val_mask     device, N bytes (nonzero = validation entry), or NULL: the
 *                held-out entries whose loss V[k] (sum of D over them, after k
 *                sweeps) is evaluated after every sweep; normally disjoint from
 *                the training mask;
 *   val_patience > 0 (with val_mask): stop after the sweep k whose V[k] exceeded
 *                V[k-1] for the val_patience-th time in a row (App. B uses 5);
 *   loss_trace   device, iters + 1 doubles, or NULL: L[0..]; entries past the
 *                stop are left untouched;
 *   val_trace    device, iters + 1 doubles, or NULL: V[0..] (needs val_mask).
 * The iteration cap is nef_fit_ctl's iters.  Each validation evaluation is one
 * more pass over Y per sweep.
 */
typedef struct {
    double tol;
    double* loss_trace;
    const uint8_t* val_mask;
    int val_patience;
    double* val_trace;
} nef_fit_control;

/*
 * nef_fit_ctl -- nef_fit under the stopping rules of *ctl (NULL = none: exactly
 * iters sweeps).  With a rule, the loop runs entirely on the device: sweeps 2..
 * are the body of a CUDA-graph conditional (while) node whose last kernel
 * applies the rules and ends the loop, so the host does not wait between
 * sweeps (with opt.eager the host reads the decision after every sweep).
 *   sweeps : host, receives the number of sweeps run, or NULL (reading it
 *            synchronises the stream; nef_plan_sweeps gives it later)
 * Errors as nef_fit, plus NEF_EINVAL for tol < 0, val_patience < 0, or
 * val_trace / val_patience without val_mask.
 */
nef_status nef_fit_ctl(nef_plan_t plan, const void* Y, const uint8_t* mask, void* const* factors, double alpha,
                       double beta, int iters, const nef_fit_control* ctl, int* sweeps);

/* Number of sweeps the last nef_fit on `plan` ran (iters unless a stopping rule
 * ended it earlier).  Synchronises the plan's stream when the count is still on
 * the device (fits with a stopping rule). */
int nef_plan_sweeps(nef_plan_t plan);

/*
 * nef_plan_autotune -- choose the column-split count (CTAs per row block) of
 * every fused pass by timing the pass kernel alone (CUDA events, median of 3)
 * for candidates of one to four waves of CTAs over the device's SMs, on the
 * given data (arguments as nef_fit; the factors are read, not changed).  With
 * cache_path, choices are looked up first in that text file (one "key<TAB>split"
 * line per pass view, precision, loss, mask and SM count) and the file is
 * rewritten with every choice.  splits (host, L ints, or NULL) receives the
 * chosen splits (-1 for passes without a fused kernel).  Synchronises the
 * plan's stream.  Errors as nef_fit, plus NEF_EINVAL for an unwritable cache.
 */
nef_status nef_plan_autotune(nef_plan_t plan, const void* Y, const uint8_t* mask, void* const* factors,
                             double alpha, double beta, const char* cache_path, int* splits);

/*
 * nef_update -- one inner step of Algorithm 1: update factor l only, with the
 * other factors held fixed.  Arguments as nef_fit; l in [0, L).
 */
nef_status nef_update(nef_plan_t plan, int l, const void* Y, const uint8_t* mask,
                      void* const* factors, double alpha, double beta);

/*
 * nef_numden -- the numerator and denominator of Eq. 3.6-3.8 for factor l at
 * the given factors (the first half of Algorithm 1's inner step), without the
 * update; for callers that sum them over shards of Y before updating (slabs of
 * Y on several GPUs: num and den are sums over the entries of Y, so the sum of
 * the slabs' num and den is the whole tensor's).
 *   num, den : device, factor l's size in the plan's element type, written
 * Arguments otherwise as nef_update.  Errors as nef_update.
 */
nef_status nef_numden(nef_plan_t plan, int l, const void* Y, const uint8_t* mask, void* const* factors,
                      double alpha, double beta, void* num, void* den);

/*
 * nef_apply_update -- the second half of the inner step: Eq. 3.4 for factor l
 * from given num and den, theta <- max(eps, theta * g^{-1}(num/den)) with g of
 * the plan's loss family (den == 0 keeps theta); refreshes the plan's operand
 * copies of factor l.  num, den: device, factor l's size.  Errors: NEF_EINVAL
 * (null pointer, factor index, alpha/beta), NEF_ECUDA.
 */
nef_status nef_apply_update(nef_plan_t plan, int l, void* const* factors, const void* num, const void* den,
                            double alpha, double beta);

/*
 * nef_loss -- sum over observed entries of D_{alpha,beta}(y, yhat) (Eq. 3.1
 * with the five-case definition of App. B), with FP64 accumulation.
 *   out : host, 2 doubles: out[0] = the sum, out[1] = the number of observed
 *         entries (so out[0]/out[1] is the mean of Sec. 6.5's metric).
 * The loss is the plan's family (nef_options.loss).  NEF_BF16 plans reconstruct
 * Yhat on the tensor cores (BF16 operands, FP32 accumulation), as the loss
 * trace of nef_fit does; the other precisions on the CUDA cores in FP32/FP64.
 * Synchronises the plan's stream.  Errors as nef_fit.
 */
nef_status nef_loss(nef_plan_t plan, const void* Y, const uint8_t* mask,
                    void* const* factors, double alpha, double beta, double* out);

/*
 * nef_plan_info -- human-readable description of the per-factor passes the
 * planner chose (row/column view, bond letters, operand sources, kernels).
 * Writes at most cap bytes (NUL-terminated) into buf (host).  Returns the
 * length the full text needs.
 */
int nef_plan_info(nef_plan_t plan, char* buf, int cap);

/*
 * nef_plan_launches -- number of kernel launches one sweep of nef_fit enqueues
 * for the given mask presence (used to report launch counts): the count taken
 * when the plan last ran or recorded a sweep of that kind, or before the first
 * such sweep the planner's estimate.
 */
int nef_plan_launches(nef_plan_t plan, int has_mask);

/*
 * nef_plan_profile -- with opt.profile set: synchronise the plan's stream and
 * return (host) the summed device time in milliseconds and the number of the
 * fused-pass launches recorded since the last reset, per kernel family:
 *   ms[0], count[0] : tensor-core (tcgen05) fused passes
 *   ms[1], count[1] : CUDA-core fused passes
 * reset != 0 clears the record afterwards.  Errors: NEF_EINVAL without
 * profiling; NEF_ECUDA from the event queries.
 */
nef_status nef_plan_profile(nef_plan_t plan, double* ms, int* count, int reset);

/*
 * nef_tc_trace -- (profiling) wait-cycle counters of the tensor-core fused pass, summed over
 * every CTA of every launch on `plan` since the last reset (plans created with
 * nef_options.profile = 2, in a library built with -DNEF_TC_TRACE=1; other builds
 * compile the counters out and leave them zero.  The counters add shared-memory
 * atomics to every tile, so timings taken with them are not representative).  out (host) receives 32 values: out[0] = summed
 * CTA lifetimes in SM cycles; out[k], k = 1..12 = cycles spent in bounded waits
 * at site k: 1 producer waits for a free Y stage, 3 MMA waits for the P tile,
 * 4 MMA waits for a Q tile, 5 MMA waits for a free yhat buffer, 6 MMA waits for
 * a W tile, 8 operand warps wait for a free Q stage, 9 epilogue waits for yhat,
 * 10 epilogue waits for Y, 11 epilogue waits for a free W buffer, 12 epilogue
 * waits for the final S, 13 operand warps wait for staged source rows, 14
 * producer waits for a free row stage; busy
 * phases: 16 operand look-ahead, 17 operand build, 18 operand fence and
 * arrival, 20 epilogue TMEM load, 21 epilogue Y read, 22 epilogue weights,
 * 23 epilogue W store, 24 epilogue fence and arrival (waits and phases of the
 * operand and epilogue warps are counted once per warp).  reset != 0 clears the counters afterwards.  Returns 0, 1 for
 * a plan without counters, 5 for a CUDA error.  Synchronises the plan's stream.
 */
int nef_tc_trace(nef_plan_t plan, unsigned long long* out, int reset);

/*
 * nef_check -- synchronise the plan's stream and report device-side errors
 * raised by earlier calls on this plan: NEF_ETIMEOUT if a bounded wait inside
 * a kernel gave up (the kernel then exits cleanly, the results of that call
 * are invalid, the context stays usable), NEF_ECUDA for an asynchronous CUDA
 * error.  Clears the device flag.
 */
nef_status nef_check(nef_plan_t plan);

/*
 * nef_fit_batched -- fit many independent CP models "ir,jr,kr->ijk" at once,
 * each from several starting points (random restarts; the paper's conclusion
 * notes that the method benefits from multiple random initializations), by
 * `iters` sweeps of Algorithm 1 per (problem, restart).  All restarts of a
 * problem share each read of its Y.  The sweep loop is captured in one CUDA
 * graph and launched once.
 *   n          : number of problems
 *   shapes     : host, n x 3 dimensions {I, J, K}
 *   ranks      : host, n ranks R (1..32)
 *   Y          : host array of n device pointers, row-major [I][J][K] floats
 *   masks      : host array of n device pointers (N bytes each, nonzero =
 *                observed), or NULL (every entry observed)
 *   factors    : host array of n*restarts*3 device pointers: for problem p and
 *                restart k, entries (p*restarts + k)*3 + {0,1,2} are A [I][R],
 *                B [J][R], C [K][R], updated in place
 *   restarts   : 1..16
 *   alpha, beta, iters : as nef_fit
 *   opt        : options (NULL = defaults); precision must be NEF_BF16
 *   losses     : host, n*restarts doubles receiving the final sum of D over
 *                observed entries per (problem, restart), or NULL
 * Work buffers (a zero-padded copy of every Y, partials, operand copies) are
 * allocated for the duration of the call.  Synchronises opt->stream.
 * Errors: NEF_EINVAL, NEF_EUNSUPPORTED (precision or (alpha, beta)), NEF_ENOMEM
 * or NEF_ECUDA (reported as NEF_ECUDA), NEF_ETIMEOUT (a bounded wait gave up).
 */
nef_status nef_fit_batched(int n, const int64_t* shapes, const int64_t* ranks, const float* const* Y,
                           const uint8_t* const* masks, float* const* factors, int restarts,
                           double alpha, double beta, int iters, const nef_options* opt,
                           double* losses);

/*
 * nef_fit_batched_tune -- the autotuner of the batched engine's work-item size:
 * times nef_fit_batched over two sweeps with each of 16, 32, 64, 128 and 256
 * column tiles per work item (nef_options.batch_tiles), on copies of the
 * factors (the caller's factors are left unchanged), and returns the fastest in
 * *tiles; ms (host, 5 doubles, or NULL) receives each candidate's wall time in
 * that order.  Arguments as nef_fit_batched.  Allocates the factor copies for
 * the duration of the call; synchronises opt->stream.  Errors as nef_fit_batched.
 */
nef_status nef_fit_batched_tune(int n, const int64_t* shapes, const int64_t* ranks, const float* const* Y,
                                const uint8_t* const* masks, float* const* factors, int restarts,
                                double alpha, double beta, const nef_options* opt, int* tiles, double* ms);

/*
 * nef_cp3_update_static -- update factor l of the 3-way CP model
 * "ir,jr,kr->ijk" in place (one inner step of the sweep, FP32, no mask)
 * without allocating any device memory.  The paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc, such as code
 * running while a framework's caching allocator owns the device memory, or
 * loops that forbid allocation after start-up.
 *   Y       : device, I*J*K floats, row-major [i][j][k]
 *   shape   : host, {I, J, K}
 *   rank    : R; must be 16, 32 or 64
 *   factors : host array of 3 device pointers: A [I][R], B [J][R], C [K][R];
 *             factor l is updated in place, the others are read
 *   alpha, beta, eps : as for nef_fit / nef_options
 *   stream  : cudaStream_t the work is ordered on
 * Intermediates live in one fixed 16 MiB device array inside the library
 * (kept by every GPU that loads it until the process exits), so the updated
 * factor must satisfy rows x R <= 1,048,576 (rows = I, J or K); larger sizes
 * return NEF_EINVAL.  Every call shares that array: calls that can overlap on
 * the GPU (other streams or host threads) race and must be serialised by the
 * caller.  Every call looks up the array's device address (so a device reset,
 * after which the array may move, is followed); the first call on a device
 * loads the library's device code there, so make it before any stream
 * capture.  The launch grid is sized from the device's SM count.  Returns
 * once the work is enqueued.
 * Errors: NEF_EINVAL (null pointer, bad rank, factor index or size, alpha or
 * beta not finite, eps negative or not finite), NEF_EUNSUPPORTED (alpha == 0
 * with beta != 1), NEF_ECUDA (launch failure).  The C entry point cannot see
 * the factors' sizes: the caller guarantees factor m has shape[m] x rank
 * floats (the Python binding checks this before the call).
 */
nef_status nef_cp3_update_static(const float* Y, const int64_t* shape, int rank,
                                 float* const* factors, int l, double alpha, double beta,
                                 double eps, void* stream);

/* Message for the last failed call on this thread ("" if none). */
const char* nef_last_error(void);

/* ------------------------------------------------------------- fold-in encoder
 * A learned initialiser for folding a new slice into a fitted 3-way CP model
 * 'ir,jr,kr->ijk' (the paper has no learned part: its fold-in of a new slice is
 * Algorithm 1's update of that slice's loading with the other factors fixed,
 * which nef_update(l = 0) performs and which refines this encoder's output).
 * The encoder is the MLP
 *     out = softplus(relu(relu(log1p(x) W1 + b1) W2 + b2) W3 + b3)
 * from one slice x = Y[i, :, :] (d_in = J*K values) to its loading row A[i, :]
 * (d_out = R values), trained on (slice, loading) pairs by Adam on
 *     L = mean over the batch and outputs of (log1p(out) - log1p(target))^2.
 * Products run on the tensor cores in BF16 with FP32 accumulation; parameters,
 * gradients and Adam moments are FP32.  Parameters are packed (device FP32) as
 * W1 [d_in x d_h], b1 [d_h], W2 [d_h x d_h], b2 [d_h], W3 [d_h x d_out], b3
 * [d_out], weights row-major [fan_in x fan_out].  All calls are ordered on the
 * encoder's stream; calls that return a loss synchronise it.
 */
typedef struct nef_foldin_s* nef_foldin_t;

/* Number of FP32 values of the packed parameters. */
int64_t nef_foldin_num_params(int d_in, int d_h, int d_out);

/*
 * nef_foldin_create -- an encoder d_in -> d_h -> d_h -> d_out for batches of at
 * most max_batch slices, starting from `params` (device, packed, copied).
 * Widths must be positive multiples of 8.  stream: cudaStream_t or NULL.
 * Errors: NEF_EINVAL, NEF_ENOMEM, NEF_ECUDA.  On error *out is NULL.
 */
nef_status nef_foldin_create(int d_in, int d_h, int d_out, int max_batch, const float* params, void* stream,
                             nef_foldin_t* out);
void nef_foldin_destroy(nef_foldin_t enc);

/*
 * nef_foldin_grad -- gradient of L at the current parameters for one batch.
 *   slices  : device [n x d_in] FP32 (raw nonnegative values; log1p is applied inside),
 *             or NULL for the batch kept by nef_foldin_load_batch
 *   targets : device [n x d_out] FP32 loadings
 *   grads   : device, packed like the parameters, receives dL/dparams
 *   loss    : host, receives L (synchronises), or NULL
 * Errors: NEF_EINVAL (n outside [1, max_batch], NULL pointer), NEF_ECUDA,
 * NEF_ETIMEOUT (a bounded wait inside a product gave up).
 */
nef_status nef_foldin_grad(nef_foldin_t enc, const float* slices, const float* targets, int n, float* grads,
                           double* loss);

/*
 * nef_foldin_load_batch -- compute the input features (log1p of the slices, in
 * BF16, and their transposed copy) of one batch of n slices once and keep them
 * in the encoder, for full-batch training: nef_foldin_grad and
 * nef_foldin_train_step with slices == NULL then use them instead of recomputing
 * them on every step (the same values, so the same results).  The kept batch
 * is dropped by any call that passes slices (including nef_foldin_predict);
 * slices == NULL without a kept batch of the same n is NEF_EINVAL.
 * Errors: NEF_EINVAL (n outside [1, max_batch], NULL pointer), NEF_ECUDA.
 */
nef_status nef_foldin_load_batch(nef_foldin_t enc, const float* slices, int n);

/*
 * nef_foldin_train_step -- forward, backward and one Adam step (Kingma & Ba,
 * bias-corrected with the encoder's step count) on one batch (slices, or NULL
 * for the batch kept by nef_foldin_load_batch); loss (host, or NULL) receives L
 * before the step.  Errors as nef_foldin_grad, plus NEF_EINVAL for lr <= 0, beta
 * outside [0, 1) or eps <= 0.
 */
nef_status nef_foldin_train_step(nef_foldin_t enc, const float* slices, const float* targets, int n, double lr,
                                 double beta1, double beta2, double eps, double* loss);

/* nef_foldin_predict -- out (device [n x d_out]) = the encoder's loadings for n slices. */
nef_status nef_foldin_predict(nef_foldin_t enc, const float* slices, int n, float* out);

/* nef_foldin_params -- copy the current packed parameters to out (device). */
nef_status nef_foldin_params(nef_foldin_t enc, float* out);

#ifdef __cplusplus
}
#endif

#endif /* NEF_H */

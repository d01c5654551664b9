/*
 * logbessel.h -- C ABI of the GB300 log-Bessel library.
 *
 * Batched, overflow-free evaluation of log I_v(x) and log K_v(x), the
 * logarithms of the modified Bessel functions of the first and second kind,
 * over many (order v, argument x) pairs, with the region-dispatched log-scale
 * algorithms of Plesner, Sorensen and Hauberg, "Accurate Computation of the
 * Logarithm of Modified Bessel Functions on GPUs" (ICS 2024, arXiv 2409.08729).
 *
 * Conventions shared by every entry point:
 *   - v, x and out are DEVICE pointers owned by the caller (for example the
 *     data pointers of CUDA tensors).  They must be valid on the current
 *     device for the duration of the enqueued work.  Element i reads
 *     v[i * v_stride] and x[i] and writes out[i]; out must not alias v or x
 *     unless it is exactly equal to x (element-wise in place is allowed).
 *   - v_stride is 1 (one order per pair) or 0 (one order for all pairs).
 *   - cuda_stream is a cudaStream_t (NULL = the legacy default stream).  Calls
 *     only enqueue work on that stream; they never synchronize.  Temporary
 *     device memory comes from the stream-ordered allocator
 *     (cudaMallocAsync) on that stream and is released on it.
 *   - n == 0 returns LB_OK without launching anything.  n < 0, a NULL pointer
 *     with n > 0, a v_stride other than 0/1, or an unknown dtype/mode returns
 *     LB_EINVAL and enqueues nothing.  Launch failures return LB_ECUDA.  The
 *     message of the last failure on the calling thread is available from
 *     logbessel_last_error().
 *   - Per-element domain results (never a status): see logbessel_i and
 *     logbessel_k.  NaN in gives NaN out.
 */
#ifndef LOGBESSEL_H
#define LOGBESSEL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LB_OK = 0,
  LB_EINVAL = 1,   /* bad argument; nothing was enqueued                     */
  LB_ECUDA = 2,    /* a CUDA call or kernel launch failed                    */
  LB_ENOMEM = 3,   /* temporary device memory could not be obtained          */
  LB_ETIMEOUT = 4, /* a bounded device-side wait gave up (serving loop)      */
  LB_ENOTSUP = 5   /* valid request that this build does not implement       */
} lb_status;

typedef enum {
  LB_F64 = 0,      /* v, x, out are double                                   */
  LB_F32 = 1       /* v, x, out are float (FP32-mixed evaluation)            */
} lb_dtype;

typedef enum {
  /* Default.  The paper's GPU expressions (mu_20, U_13, power series or
   * integral) with region thresholds moved so that the truncation error of
   * each expression stays below 3e-16 of the error scale, and Gauss
   * quadrature in place of Simpson's rule for the K integral. */
  LB_TIGHT = 0,
  /* The paper's GPU algorithm as printed: Algorithm 1 without the mu_3, U_4,
   * U_6, U_9 branches (Sec. 4.3), Table "input ranges" thresholds, composite
   * Simpson with N = 600 and the heuristic maxima for the K integral
   * (Sec. 3.2), with the Simpson constant read as 1/(3N). */
  LB_PAPER_GPU = 1,
  /* Algorithm 1 in the paper's CPU order (all seven branches). */
  LB_PAPER_CPU_ORDER = 2
} lb_mode;

/* Region ids written by logbessel_classify (Table "input ranges"). */
typedef enum {
  LB_R_MU20 = 0,      /* large-argument expansion, 20 terms (Eqs. "log Iv mu k", "log Kv mu k") */
  LB_R_U13 = 1,       /* uniform large-order expansion, 13 terms (Eqs. "log Iv u k", "log Kv u k") */
  LB_R_FALLBACK = 2,  /* power series for I (Eq. "log Iv"), integral for K (Eq. "log Kv integral") */
  LB_R_SPECIAL = 3,   /* domain edge: NaN, zero or infinite input, negative order for I */
  LB_R_MU3 = 4,       /* the remaining expressions of the CPU order */
  LB_R_U4 = 5,
  LB_R_U6 = 6,
  LB_R_U9 = 7
} lb_region;

/*
 * log I_v(x), the modified Bessel function of the first kind, for v >= 0,
 * x >= 0 (paper Sec. 3.1; Algorithm 1).
 *   v < 0 or x < 0 -> NaN;  x = 0 -> 0 if v = 0, else -inf;
 *   x = +inf (v finite) -> +inf;  v = +inf (x finite) -> -inf;
 *   v and x both infinite -> NaN.
 */
lb_status logbessel_i(lb_dtype dtype, const void* v, int64_t v_stride, const void* x, void* out,
                      int64_t n, lb_mode mode, void* cuda_stream);

/*
 * log K_v(x), the modified Bessel function of the second kind, for real v
 * (K_{-v} = K_v, so |v| is used) and x >= 0 (paper Sec. 3.2; Algorithm 1).
 *   x < 0 -> NaN;  x = 0 -> +inf;  x = +inf (v finite) -> -inf;
 *   v = +-inf (x finite, > 0) -> +inf;  v and x both infinite -> NaN.
 */
lb_status logbessel_k(lb_dtype dtype, const void* v, int64_t v_stride, const void* x, void* out,
                      int64_t n, lb_mode mode, void* cuda_stream);

/*
 * Caller-supplied workspace.  The K entry points queue the pairs that take
 * the integral (the fallback region) in device scratch: 256 bytes for a
 * counter and the mask of the quadrature rules queued, plus 4 bytes per pair
 * of a pass.  logbessel_k and logbessel_k_dx
 * take it from the stream-ordered allocator; these variants take it from the
 * caller and allocate nothing.
 *
 * logbessel_workspace_bytes(n): the bytes that evaluate n pairs in one pass,
 * 256 + 4 min(m, 2^26) with m = n rounded up to a multiple of 2048 (the
 * tile of the per-call kernels), at least 8448 (0 for n < 0).
 * logbessel_k_ws / logbessel_k_dx_ws: as logbessel_k / logbessel_k_dx, with
 * `workspace` a device pointer (256-byte aligned) to `ws_bytes` bytes, at
 * least 8448 (2048 pairs per pass); n pairs are processed in passes of
 * (ws_bytes - 256) / 4 pairs rounded down to a multiple of 2048 (at most
 * 2^26), with results identical to one pass.  The workspace is used in
 * stream order on cuda_stream: other work must not use it until the call's
 * work has finished.  LB_EINVAL (nothing enqueued) for a NULL, misaligned
 * or too small workspace; other errors as the plain entry points.
 */
int64_t logbessel_workspace_bytes(int64_t n);
lb_status logbessel_k_ws(lb_dtype dtype, const void* v, int64_t v_stride, const void* x, void* out, int64_t n,
                         lb_mode mode, void* workspace, int64_t ws_bytes, void* cuda_stream);
lb_status logbessel_k_dx_ws(lb_dtype dtype, const void* v, int64_t v_stride, const void* x, void* out, int64_t n,
                            lb_mode mode, void* workspace, int64_t ws_bytes, void* cuda_stream);

/*
 * log K_v(x) like logbessel_k (FP64 only), but without allocating any device
 * memory.  The paper has no counterpart: this entry point exists for callers
 * that cannot let a library allocate, such as code that runs under a device
 * memory budget fixed in advance, latency-critical loops where an allocation
 * may block or fail at the wrong moment, or frameworks whose own allocator
 * must own all device memory.
 *
 * The K fallback pairs are queued in a fixed scratch array that the library
 * defines in device global memory: 4 MiB plus 256 bytes, resident on every
 * GPU that loads the library until the process exits.  Hence at most
 * 1048576 pairs per call; a larger n returns LB_EINVAL with a message and
 * launches nothing.  Every call looks up the scratch address
 * (cudaGetSymbolAddress, no allocation) in the current context, so the entry
 * point stays valid after cudaDeviceReset; the first call on a device may
 * load the library's module, so make it before any stream capture on that
 * device.  Every call shares the one
 * array and clears its counter and mask on the stream: calls whose work overlaps on
 * the GPU (different streams, or concurrent host threads) race and must be
 * serialized by the caller.  Other arguments, results and errors as in
 * logbessel_k; LB_ENOTSUP for LB_F32.
 */
lb_status logbessel_k_noalloc(lb_dtype dtype, const void* v, int64_t v_stride, const void* x, void* out,
                              int64_t n, lb_mode mode, void* cuda_stream);

/*
 * d/dx log I_v(x) = I'_v(x) / I_v(x) and d/dx log K_v(x) = K'_v(x) / K_v(x):
 * the adjoint of logbessel_i / logbessel_k, computed by differentiating each
 * region's expression term by term with the same dispatch (the paper lists
 * derivatives as future work, Sec. 7; the integrand derivative of the K
 * integral is dF/dx = F (2v - 1)/(s + 2x)).  Same arguments as logbessel_i.
 * Domain edges: x = 0 gives 0 (I, v = 0), +inf (I, v > 0), -inf (K);
 * x = +inf gives +1 (I) and -1 (K); infinite or NaN order gives NaN.
 * logbessel_k_dx supports LB_TIGHT only (LB_ENOTSUP otherwise).
 */
lb_status logbessel_i_dx(lb_dtype dtype, const void* v, int64_t v_stride, const void* x, void* out,
                         int64_t n, lb_mode mode, void* cuda_stream);
lb_status logbessel_k_dx(lb_dtype dtype, const void* v, int64_t v_stride, const void* x, void* out,
                         int64_t n, lb_mode mode, void* cuda_stream);

/*
 * von Mises-Fisher log-normaliser in dimension d (paper Sec. 6.3):
 *   deriv = 0:  log C_d(k) = (d/2 - 1) log k - (d/2) log(2 pi) - log I_{d/2-1}(k)
 *   deriv = 1:  d/dk log C_d(k) = (d/2 - 1)/k - I'_{d/2-1}(k) / I_{d/2-1}(k)
 * for every kappa[i] >= 0 (device array of n doubles), written to out[i].
 * k = 0 gives the limit lgamma(d/2) - log 2 - (d/2) log pi (deriv: 0);
 * k < 0 or NaN gives NaN.  d must be finite and >= 2 (LB_EINVAL otherwise).
 * Uses LB_TIGHT evaluation; dtype must be LB_F64.
 */
lb_status logbessel_vmf_log_c(lb_dtype dtype, double d, const void* kappa, void* out, int64_t n,
                              int deriv, void* cuda_stream);

/*
 * The same evaluations on HOST buffers, end to end: fn = 0 log I, 1 log K,
 * 2 d/dx log I, 3 d/dx log K.  v, x, out are host pointers (pinned memory
 * lets the copies overlap with the computation; pageable memory works but
 * copies synchronously).  The pairs are processed in chunks of `chunk`
 * (0 = 16M pairs; at most 2^26) through four device chunk slots and three
 * internal streams, so the copy-in of one chunk, the evaluation of the
 * previous one and the copy-out of the one before overlap; when chunk is a
 * multiple of 16384 the first and last pieces are smaller (down to chunk/8)
 * to shorten the unoverlapped copies, with results equal to one pass.  The call
 * returns when every result is in `out` (it synchronizes).  The streams,
 * events and one device buffer (four chunk slots of v, x and out, plus the
 * K fallback queue: about 4 * 24 * chunk + 4 * chunk bytes in FP64) belong to the
 * current device and are kept from one call to the next, grown when a call
 * needs more; calls on the same device run one at a time (a lock).
 * Errors as for the device entry points; LB_ENOTSUP for derivatives in FP32
 * or the K derivative outside LB_TIGHT; LB_ENOMEM when the buffer cannot be
 * allocated.
 */
lb_status logbessel_host(int fn, lb_dtype dtype, const void* v, int64_t v_stride, const void* x, void* out,
                         int64_t n, lb_mode mode, int64_t chunk);

/*
 * Release the streams, events and device buffer that logbessel_host keeps
 * for the current device (after waiting for its streams).  The next
 * logbessel_host call on that device creates them again.  Returns LB_OK, or
 * LB_ECUDA when the current device cannot be read.
 */
lb_status logbessel_host_release(void);

/*
 * Region id of every pair under the dispatch of `mode` (Table "input
 * ranges"; Algorithm 1 and the GPU subset of Sec. 4.3).  kind = 0 for I,
 * 1 for K (K classifies |v|).  region_out is a device array of n uint8_t.
 */
lb_status logbessel_classify(int kind, lb_dtype dtype, const void* v, int64_t v_stride,
                             const void* x, uint8_t* region_out, int64_t n, lb_mode mode,
                             void* cuda_stream);

/*
 * Evaluate ONE expression for every pair, bypassing the dispatch: region is
 * an lb_region value (MU20, U13, FALLBACK, or with LB_PAPER_CPU_ORDER also
 * MU3, U4, U6, U9).  For checking each expression on both sides of a region
 * boundary.  Domain edges still give the values listed above.  `mode` selects
 * the quadrature of the K integral (Gauss for LB_TIGHT, Simpson otherwise).
 */
lb_status logbessel_eval_region(int kind, lb_dtype dtype, const void* v, int64_t v_stride,
                                const void* x, void* out, int64_t n, int region, lb_mode mode,
                                void* cuda_stream);

/*
 * Kernel accounting (tracing).  Every kernel launch the library makes is
 * counted; with profiling enabled each launch is also bracketed by two CUDA
 * events recorded on its stream, and logbessel_profile_get sums the elapsed
 * times per kernel.  Enabling resets the timers.  logbessel_profile_get waits
 * for the recorded events (it synchronizes with the timed launches).
 * slot: 0 = lb_tiles_kernel, 1 = lb_kint_kernel, 2 = lb_classify_kernel,
 * 3 = small auxiliary kernels (logbessel_profile_slots() gives the count).  *name points to a static
 * string.  Returns LB_EINVAL for a slot out of range.
 */
void logbessel_profile_enable(int on);
int logbessel_profile_slots(void);
lb_status logbessel_profile_get(int slot, const char** name, long long* launches,
                                long long* timed_launches, double* total_ms);
/* Total kernel launches made by this library in this process. */
long long logbessel_launch_count(void);

/*
 * Measure the FP64-pipe roofline of the current GPU (microbenchmarks with
 * every SM busy; runs about 0.2 s and synchronizes the stream).  rates is a
 * host array of 13 doubles that receives operations per second for: DFMA,
 * exp, log, division, sqrt, lgamma (CUDA, double precision), and the
 * library's table-driven exp and log, its exp for quadrature terms (no low
 * table part), and its integer-pipe exp, log, reciprocal and 1/sqrt (13
 * doubles in all).
 * Returns LB_EINVAL for
 * a NULL rates, LB_ENOMEM or LB_ECUDA on failure.
 */
lb_status logbessel_measure_fp64(double* rates, void* cuda_stream);

/*
 * Elementwise double-precision exp/log used inside the kernels, exposed for
 * checking: which = 0 table-driven exp, 1 table-driven log (Tang's method),
 * 2 CUDA exp, 3 CUDA log, 4 log(cyl_bessel_i0), 5 log(cyl_bessel_i1) (CUDA's
 * order-0/1 functions, the comparison system of paper Sec. 6.1), 6 the
 * table-driven exp without the low table part (quadrature terms; y <= 708),
 * 7 exp, 8 log, 9 reciprocal and 10 1/sqrt in fixed-point integer
 * arithmetic (exp: y <= 708), 11 the Q53 log (out holds the int64 result's
 * bits) and 12 the Q58 exponential of a Q53 shift d <= 0 (in holds d's
 * int64 bits, out the uint64 result's bits), the K integral's node
 * functions.  in/out are device arrays of n doubles (8-byte words).
 * LB_EINVAL for a bad which, size or pointer.
 */
lb_status logbessel_math_eval(int which, const double* in, double* out, int64_t n, void* cuda_stream);

/*
 * Continuous-batching server (serving loop).  Requests of any size arrive
 * from host threads; a scheduler thread admits them as request slots and
 * device memory (a fixed arena) free up, copies the inputs of host requests
 * to the GPU, and publishes their work to a persistent kernel, which
 * interleaves the work of all resident requests, so requests that arrive
 * while others run overlap on the device.  A request runs the two stages of
 * a direct call: tiles (classify, bin, expressions), then for log K the
 * integral of the fallback pairs, queued per quadrature rule class and
 * evaluated in windows of one class each (paper Sec. 3.2; Sec. 4.3 groups
 * pairs by expression for the same reason: one code path per warp).
 * Results of host requests are copied back into the caller's buffer.
 *
 *   arena_bytes  device memory for request buffers (>= 1 MiB); a host
 *                request needs 3 n elements (v, x, out), a log K request
 *                also its queues: 24 n bytes (FP64, LB_TIGHT: six rule
 *                classes) or 4 n bytes; each part rounded to 256 B
 *   max_slots    requests resident on the device at once (1..4096)
 *   ctas_per_sm  persistent thread blocks per SM (1..8)
 *   idle_ms      a thread block with no work for this long exits; the
 *                scheduler relaunches the kernel when work appears (every
 *                device-side wait is bounded by it)
 *
 * The server runs on the device current at lb_server_create.  v, x, out of
 * lb_server_submit are HOST pointers (pinned memory lets the copies overlap
 * with computation); they must stay valid until lb_server_wait returns LB_OK
 * for the ticket.  kind 0 = log I, 1 = log K; dtype LB_F64 or LB_F32
 * (FP32-mixed; FP32 K requires LB_TIGHT).  Requests larger than the arena
 * are rejected with LB_ENOMEM; bad arguments with LB_EINVAL (nothing queued).
 * lb_server_wait returns LB_ETIMEOUT if the result is not ready in time (the
 * request stays queued).  Times from lb_server_ticket_info are seconds on a
 * monotonic clock: submission, admission (copy-in started) and completion
 * (result in the host buffer).  lb_server_release forgets a finished ticket.
 * lb_server_destroy stops the kernel and frees everything.  The paper has no
 * serving component; this is the batched front end of the same kernels.
 *
 * lb_server_submit_device: the same request on DEVICE buffers v, x, out of
 * the server's device; nothing is copied and the results are written to out
 * in place.  The inputs must be complete when the request is admitted: pass
 * a cudaEvent_t recorded after the work that writes them as ready_event (the
 * server starts the request once the event has completed; the event must
 * stay valid until lb_server_wait returns LB_OK), or NULL when they are
 * already complete.  When lb_server_wait returns LB_OK the results are in
 * out and the server no longer reads v and x.  The arena then holds only the
 * K queues (none for log I).
 */
typedef struct lb_server lb_server;
typedef struct {
  int64_t arena_bytes;
  int max_slots;
  int ctas_per_sm;
  double idle_ms;
} lb_server_config;

lb_status lb_server_create(const lb_server_config* cfg, lb_server** server);
lb_status lb_server_submit(lb_server* server, int kind, lb_dtype dtype, const void* v, int64_t v_stride,
                           const void* x, void* out, int64_t n, lb_mode mode, long long* ticket);
lb_status lb_server_submit_device(lb_server* server, int kind, lb_dtype dtype, const void* v, int64_t v_stride,
                                  const void* x, void* out, int64_t n, lb_mode mode, void* ready_event,
                                  long long* ticket);
lb_status lb_server_wait(lb_server* server, long long ticket, double timeout_s);
lb_status lb_server_ticket_info(lb_server* server, long long ticket, int* done, double* t_submit,
                                double* t_admit, double* t_done);
lb_status lb_server_release(lb_server* server, long long ticket);
lb_status lb_server_stats(lb_server* server, long long* completed, long long* evals,
                          long long* kernel_launches, long long* in_flight);
/*
 * Device time accounts of the persistent kernel, cumulative since
 * lb_server_create (take differences between two reads).  claim_ns: the
 * summed time its CTAs spent claiming a work item, waiting for one included
 * (a CTA with nothing to do counts here until it exits).  busy_ns[f] and
 * items[f], f < LB_SERVER_FAMILIES: the summed time CTAs spent running the
 * items of family f, and how many ran; the families are 0 FP64 log I tiles,
 * 1 FP64 log K tiles, 2 FP32 log I tiles, 3 FP32 log K tiles, 4 + c the
 * windows of the FP64 K-integral queue of rule class c (c < 6; the paper
 * modes' single queue counts as class 0), 10 FP32 K-integral windows.  Times
 * are ns of the device's global timer.  The counters are read by a copy on a
 * stream of the server's own while the kernel runs; the call blocks until
 * that copy is done.  Any pointer may be NULL.  LB_ECUDA if the copy fails.
 */
#define LB_SERVER_FAMILIES 11
lb_status lb_server_device_stats(lb_server* server, long long* claim_ns, long long* busy_ns,
                                 long long* items);
lb_status lb_server_destroy(lb_server* server);
/* Message describing the last server failure on the calling thread. */
const char* lb_server_last_error(void);

/*
 * Index checks (the checked build, compiled with LB_CHECKS into
 * liblogbessel_checks.so).  There, every index into a tile's shared list,
 * into the K-integral queue, and every pair offset read back from the queue
 * is checked against its bound before use; a failed check sets a bit of a
 * device status word (1 list write, 2 list read, 4 queue write, 8 queue
 * count above the capacity, 16 pair offset beyond the chunk, 32 rule class
 * out of range) and the access is skipped, so an index error is recorded
 * instead of faulting.  Results are identical to the release build's when
 * no check fails.  logbessel_check_status stores the word in *bits (host
 * pointer) and clears it when clear != 0; it synchronizes the device.
 * Release builds: *bits = 0 and LB_ENOTSUP.  The paper has no counterpart.
 */
lb_status logbessel_check_status(unsigned int* bits, int clear);

/* Message describing the last failure on the calling thread ("" if none). */
const char* logbessel_last_error(void);

/* Library version string. */
const char* logbessel_version(void);

#ifdef __cplusplus
}
#endif

#endif /* LOGBESSEL_H */

/*
 * fft2d.h -- C ABI of a GB300 (sm_103a) library for the 2D forward and
 * inverse complex FFT of an image by radix-2 decimation in time.
 *
 * Method (Shen et al., "Research on the fast Fourier transform of image
 * based on GPU"):
 *   - Section 2, eq. 1: X(k) = sum_{n<N} x(n) W_N^{nk}.
 *   - Section 2, eqs. 2-3: the radix-2 DIT recurrence X(k) = Xe(k) + W_N^k Xo(k),
 *     X(k+N/2) = Xe(k) - W_N^k Xo(k), applied over log2(N) stages of N/2
 *     independent butterflies.
 *   - Section 3.1, eq. 4: the butterfly X(k) = X1(k) + W * X2(k), with
 *     rotation factors precomputed once per size.
 *   - Section 3.2: a bit-reversal scramble before the stages, so that they
 *     run in place; 2D = every row, then every column, each axis scrambled
 *     along itself.
 *
 * Conventions (readings of points the paper leaves open):
 *   - W_N = exp(-2*pi*i/N) forward, exp(+2*pi*i/N) inverse.
 *   - Forward unscaled, inverse multiplied by 1/(rows*cols).
 *   - Rows first, then columns.
 *
 * Data layout: a rows x cols image is row-major, with interleaved complex
 * values: FFT2D_C64 is (float re, float im), 8 bytes per pixel, the layout of
 * torch.complex64 / numpy.complex64.
 *
 * Ownership: image buffers (device or host) belong to the caller.  A plan
 * owns its device twiddle tables and any staging buffer it allocates; all of
 * them are released by fft2d_destroy.  Every fft2d_exec* call is
 * asynchronous on the given CUDA stream (NULL = the legacy default stream)
 * except where noted.
 *
 * Errors: argument errors are returned synchronously and nothing is
 * launched.  A launch failure returns FFT2D_ERR_CUDA; fft2d_last_error()
 * gives the CUDA error text of the calling thread's last failure.  Calls must
 * be made with the plan's device current.
 */
#ifndef FFT2D_H
#define FFT2D_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define FFT2D_API __attribute__((visibility("default")))
#else
#define FFT2D_API
#endif

typedef struct fft2d_plan_s *fft2d_plan_t;

/* Storage types (dtype argument). */
#define FFT2D_C64 0  /* complex64: float2 per pixel, FP32 arithmetic */
#define FFT2D_C32H 1 /* half2 per pixel + a power-of-two exponent per line, FP32 arithmetic */
#define FFT2D_R32_DCT2 2 /* real float per pixel: the 2D DCT-II (see fft2d_plan), FP32 arithmetic */

/* Directions (dir argument). */
#define FFT2D_FORWARD (-1)
#define FFT2D_INVERSE 1

/* Passes (fft2d_exec_pass). */
#define FFT2D_PASS_ROWS 0
#define FFT2D_PASS_COLS 1

/* Largest side accepted (2^14). */
#define FFT2D_MAX_SIDE 16384

typedef enum {
    FFT2D_OK = 0,
    FFT2D_ERR_ARG = 1,         /* null pointer, bad enum, bad stage count   */
    FFT2D_ERR_NOT_POW2 = 2,    /* a side is not a power of two (or < 1)     */
    FFT2D_ERR_TOO_LARGE = 3,   /* a side exceeds FFT2D_MAX_SIDE             */
    FFT2D_ERR_OOM = 4,         /* device or host allocation failed          */
    FFT2D_ERR_CUDA = 5,        /* a CUDA call or launch failed              */
    FFT2D_ERR_TIMEOUT = 6,     /* a bounded device wait ran out             */
    FFT2D_ERR_BUDGET = 7,      /* request does not fit the memory budget    */
    FFT2D_ERR_UNSUPPORTED = 8  /* valid but not provided by this build      */
} fft2d_status;

/*
 * Create a plan for a rows x cols transform (1 <= side <= FFT2D_MAX_SIDE,
 * powers of two; 1 means that axis is left unchanged).  Builds the per-stage
 * rotation-factor tables of both axes on the host in FP64 (Section 3.1:
 * "calculated in advance ... not changed") and uploads them, rounded to FP32,
 * to the current device.  *out receives the plan; on error it is set to NULL.
 */
FFT2D_API fft2d_status fft2d_plan(int rows, int cols, int dtype, int dir, fft2d_plan_t *out);

/*
 * Plans of dtype FFT2D_R32_DCT2: the 2D discrete cosine transform, which
 * Section 5 names as a transform the method carries over to.  The image is
 * real, one float per pixel, row-major (pitch = cols); fft2d_exec and
 * fft2d_exec_pass (rows: in -> out, columns: in -> out; in may equal out)
 * compute, with dir = FFT2D_FORWARD, the unnormalised DCT-II
 *   X[k][l] = sum_{m<rows} sum_{n<cols} x[m][n] cos(pi k (2m+1) / (2 rows))
 *                                               cos(pi l (2n+1) / (2 cols))
 * and with dir = FFT2D_INVERSE its exact inverse, the DCT-III
 *   x[m][n] = 1/(rows cols) sum_k sum_l e_k e_l X[k][l] cos(..) cos(..),
 *   e_0 = 1, e_k = 2 (k > 0),
 * as one pass along the rows, then one along the columns (whose pass
 * carries the whole 1/(rows cols), as for the FFT), each on the radix-2
 * engine: a length-N DCT-II is one length-N complex DFT of the reordered
 * line (even samples ascending, odd samples descending) followed by a
 * rotation by exp(-i pi k / (2N)) (Makhoul, 1980); the inverse rotates
 * first, then runs the inverse DFT and undoes the reordering.  Two real
 * lines share one complex line, except in the inverse column pass of 16384
 * rows, and in the forward one when cols is not a multiple of 8: there each
 * real column is its own complex line and the pass runs in place (called
 * out of place it first copies `in` to `out` on the stream).  The plan also
 * holds the
 * (cos, sin)(pi k / (2N)) tables, built in FP64 and rounded to FP32.
 * Errors: FFT2D_ERR_UNSUPPORTED for a side of 1.  The other entry points
 * reject these plans with FFT2D_ERR_ARG, except fft2d_exec_host,
 * fft2d_exec_host_many(_async), fft2d_selftest_withheld_load,
 * fft2d_plan_info, fft2d_plan_describe, fft2d_sync_status and fft2d_destroy.
 */

/*
 * Wait for all work on the device, then report device-side failures of this
 * plan's kernels since the last call: FFT2D_ERR_TIMEOUT when a bounded wait
 * inside a kernel (a TMA transfer that never completed) gave up, in which
 * case that launch's output is incomplete.  Clears the status.  A CUDA error
 * of the context is returned as FFT2D_ERR_CUDA.
 */
FFT2D_API fft2d_status fft2d_sync_status(fft2d_plan_t plan);

/*
 * Self-test of the device failure path: one small kernel waits on an mbarrier
 * phase that nothing completes, gives up after about 20 ms with the same
 * bounded wait the TMA pipeline uses, and records the timeout in the plan's
 * status word, which the next fft2d_sync_status reports as FFT2D_ERR_TIMEOUT.
 * Touches no image data and leaves the context usable.  Asynchronous.
 */
FFT2D_API fft2d_status fft2d_selftest_timeout(fft2d_plan_t plan, void *stream);

/*
 * Self-test of the failure path of the persistent TMA-fed column kernels
 * (the tile pipeline that brings each column tile of Section 2's second 1D
 * transform into shared memory): runs the plan's column pass over `in` into
 * `out` (device images of the plan's shape and dtype, row pitch = cols;
 * for FFT2D_R32_DCT2 plans the DCT column pass of the plan's direction,
 * which is TMA-fed for columns of 2048 to 16384 points), except that CTA 0
 * never issues the second TMA load of its
 * first tile.  That CTA's bounded wait gives up after about one second, the
 * kernel records the timeout -- for the cluster kernels of 8192- and
 * 16384-row columns every CTA of the cluster learns of it at the tile's
 * first cluster barrier and they leave together -- lets
 * the transfers in flight land, releases what it holds and returns; the
 * next fft2d_sync_status reports FFT2D_ERR_TIMEOUT and `out` is incomplete.
 * No GPU fault is involved and the context stays usable.
 * Errors: FFT2D_ERR_ARG for a null plan or pointer, a half2 plan, a plan with
 * one row, or when the column pass this plan would run (its variant, or the
 * default for its size, after the alignment checks) is not a TMA-fed kernel
 * (for a DCT plan: columns of other lengths, or a width that is not a whole
 * number of tiles).
 * Asynchronous on `stream`.
 */
FFT2D_API fft2d_status fft2d_selftest_withheld_load(fft2d_plan_t plan, const void *in, void *out,
                                                    void *stream);

/*
 * Autotuner.  Times every kernel variant usable for this plan's shape on the
 * current device -- per pass: CTA tile shape (rows or adjacent columns per
 * CTA), values per thread, TMA-fed persistent or plain launches, and for
 * long columns the cluster split -- on two scratch images it allocates for
 * the call, and keeps the fastest for this plan.  The choice is also kept in
 * a process-wide table (device, pass, axis length, line count) that later
 * fft2d_plan calls of the same shape pick up, and, when the environment
 * variable FFT2D_TUNE_CACHE names a file, written there and read back by
 * later processes.  Every variant computes identical results (the same
 * butterflies in the same order); only the speed differs.  Synchronous.
 */
FFT2D_API fft2d_status fft2d_autotune(fft2d_plan_t plan, void *stream);

/*
 * Write a NUL-terminated description of the kernel variant each pass of the
 * plan uses ("rows:<name>(shape=..,ept=..,tuned|default) cols:...") into
 * buf[0..len).
 */
FFT2D_API fft2d_status fft2d_plan_describe(fft2d_plan_t plan, char *buf, int len);

/* Number of kernel variants of one pass (FFT2D_PASS_ROWS/COLS) over lines of
 * 2^L points (1 <= L <= 14; 0 otherwise), and the name of variant `index`
 * ("" when out of range).  Variant 0 ("plain") serves every call. */
FFT2D_API int fft2d_variant_count(int pass, int L);
FFT2D_API const char *fft2d_variant_name(int pass, int L, int index);

/* Force the kernel variant of one pass of a plan (-1: the per-size default).
 * A variant that cannot serve a particular call (unaligned buffers, partial
 * tiles) falls back to the plain kernel for that call. */
FFT2D_API fft2d_status fft2d_plan_set_variant(fft2d_plan_t plan, int pass, int variant);

/* Release a plan and everything it owns.  NULL is accepted (no-op). */
FFT2D_API fft2d_status fft2d_destroy(fft2d_plan_t plan);

/* Report the parameters a plan was created with (any pointer may be NULL). */
FFT2D_API fft2d_status fft2d_plan_info(fft2d_plan_t plan, int *rows, int *cols, int *dtype, int *dir);

/*
 * Whole 2D transform on device buffers: the row pass (scramble fused into the
 * load, all log2(cols) stages in one launch), then the column pass (scramble
 * fused, all log2(rows) stages, inverse scale fused into the store).
 * in and out are device pointers to rows*cols pixels; in == out is allowed
 * (in place).  Partial overlap of in and out is not allowed.  Two launches.
 * Once the plan has run on its device (the first launch of each kernel sets
 * its shared-memory limit), the call may be captured in a CUDA graph on
 * `stream`.  It makes no allocation then, except that the column pass of
 * 8192 or 16384 rows (and the DCT column passes of 16384 rows and the
 * forward one of 8192 rows) takes a scratch block (about 20 to 50 MB) for the exchange
 * between the CTAs of a cluster stream-ordered from the library's own
 * device memory pool and returns it on `stream` after the launch
 * (cudaMallocFromPoolAsync / cudaFreeAsync: no device synchronisation; the
 * pool keeps its memory, so after the first calls no driver allocation
 * happens; under capture the two become graph memory nodes).  Calls on
 * different streams therefore never share scratch.
 */
FFT2D_API fft2d_status fft2d_exec(fft2d_plan_t plan, const void *in, void *out, void *stream);

/*
 * One of the two passes of fft2d_exec: FFT2D_PASS_ROWS reads `in` and writes
 * `out`; FFT2D_PASS_COLS reads `in` and writes `out` and applies the inverse
 * scale.  fft2d_exec(p, x, y) == pass(ROWS, x, y) then pass(COLS, y, y).
 * One launch.
 */
FFT2D_API fft2d_status fft2d_exec_pass(fft2d_plan_t plan, int pass, const void *in, void *out,
                             void *stream);

/*
 * Debug view of partial execution: like fft2d_exec, but each axis stops
 * after row_stages (0..log2 cols) and col_stages (0..log2 rows) butterfly
 * stages, leaving the data in the scrambled position order that the
 * in-place stages use.  With 0 stages an axis is only scrambled (Section 3.2),
 * an exact permutation.  The inverse scale is applied only when both axes run
 * every stage.  Two launches.
 */
FFT2D_API fft2d_status fft2d_exec_stages(fft2d_plan_t plan, const void *in, void *out, int row_stages,
                               int col_stages, void *stream);

/*
 * Whole transform of HOST buffers (the paper's upload / render / read-back
 * cycle, Section 1.1): copies in_host to a plan-owned device buffer
 * (allocated on first use), runs fft2d_exec in place there, copies the
 * result to out_host and waits for the stream.  Synchronous.  Pinned host
 * memory gives the full copy bandwidth; pageable memory is accepted.
 * in_host == out_host is allowed.
 */
FFT2D_API fft2d_status fft2d_exec_host(fft2d_plan_t plan, const void *in_host, void *out_host,
                             void *stream);

/*
 * fft2d_exec_host for n images at once, pipelined: while image i is
 * transformed, image i+1 uploads and image i-1 downloads, on two internal
 * copy streams and the caller's stream (six device image buffers per
 * device, grown to the largest image and kept for the life of the process).
 * Image i is transformed with plans[i] from in_host[i] to out_host[i];
 * in_host[i] == out_host[i] is allowed.  An image may read the output of an
 * earlier image of the same call (in_host[i] == out_host[j], j < i, the same
 * pointer): its upload waits for that download, so a forward transform and
 * its inverse can travel in one call.  When that earlier image is the one
 * just before (in_host[i] == out_host[i-1], images of the same byte size),
 * image i is transformed straight from the device copy of that output and
 * nothing is uploaded for it.  If image i also writes the same host buffer
 * (out_host[i] == out_host[i-1], e.g. a forward transform and its inverse in
 * place), the earlier result could never be observed on the host and is not
 * copied back; every other result is.
 * Otherwise the host buffers of
 * different images must not overlap.  The copies start after the work
 * already queued on `stream`.  complex64 and DCT plans (FFT2D_R32_DCT2,
 * 4-byte pixels) of one device only; both kinds may be mixed in one call.
 * Synchronous: every copy has finished on return, after a failure too.
 * Pinned host memory gives the full copy bandwidth (the NVLink-C2C host link
 * of a GB300 moved about 210 GB/s up, 190 GB/s down, 340 GB/s both at once).
 */
FFT2D_API fft2d_status fft2d_exec_host_many(int n, const fft2d_plan_t *plans,
                                            const void *const *in_host, void *const *out_host,
                                            void *stream);

/*
 * fft2d_exec_host_many without the final wait: returns once everything is
 * queued, with `stream` ordered after every copy and transform of the call,
 * so calls issued back to back keep the host link busy across call
 * boundaries and one synchronisation of `stream` (or an event recorded on
 * it) covers them all.  The host buffers must stay valid, and must be
 * neither written (inputs) nor read (outputs) by the host, until then.
 * Dependencies are tracked within a call only: a later call may read a host
 * buffer an earlier unfinished call writes only if that buffer is also
 * written by the later call before it reads it (as when every call carries
 * both a forward transform and its inverse).  On an error the call waits
 * for what it queued and returns the status.
 */
FFT2D_API fft2d_status fft2d_exec_host_many_async(int n, const fft2d_plan_t *plans,
                                                  const void *const *in_host,
                                                  void *const *out_host, void *stream);

/*
 * n independent transforms, possibly of different plans (sizes, directions),
 * issued on one stream: image i is transformed with plans[i] from in[i] to
 * out[i] (device pointers; in[i] == out[i] allowed; different images must not
 * overlap).  Images are grouped by axis length and direction: one launch per
 * group runs the row pass of all its images (a job table travels as a kernel
 * parameter), then one launch per group the column pass -- a handful of
 * launches for any number of images.  Lines of 8192 and 16384 points run
 * each image's single-image pass instead (the cluster column kernels), on
 * the group's internal stream.  Every image's result is bit for bit the one
 * fft2d_exec gives.  complex64 plans only.
 */
FFT2D_API fft2d_status fft2d_exec_batched(int n, const fft2d_plan_t *plans, const void *const *in,
                                void *const *out, void *stream);

/*
 * Half2 storage (plans created with FFT2D_C32H, sides >= 2).  A pixel is
 * stored as q = (re, im) in IEEE half precision, and its value is q * 2^e
 * where e is an int exponent shared by its whole row or whole column.  Each
 * pass computes in FP32 (the same butterflies and rotation factors as the
 * complex64 path) and, for every line it writes, picks e from the line's
 * largest component magnitude M = f 2^k (f in [0.5, 1)) as e = k - 14, so
 * that every stored |q| < 2^14.  Global traffic is half that of complex64.
 *
 * in: rows*cols half2 with exponents in_exp, one per row (in_axis =
 * FFT2D_PASS_ROWS) or one per column (in_axis = FFT2D_PASS_COLS).
 * out: rows*cols half2 (in == out allowed) with exponents written to
 * out_exp, one per COLUMN (the column pass owns whole columns).  The row
 * pass's per-row exponents live in the plan.  Asynchronous.
 */
FFT2D_API fft2d_status fft2d_exec_h16(fft2d_plan_t plan, const void *in, const int *in_exp,
                                      int in_axis, void *out, int *out_exp, void *stream);

/* complex64 -> half2 with one exponent per row (same rule as the passes);
 * out_exp receives `rows` ints.  Device buffers, asynchronous. */
FFT2D_API fft2d_status fft2d_h16_pack(int rows, int cols, const void *in, void *out,
                                      int *out_exp, void *stream);

/* half2 + exponents (one per row for axis FFT2D_PASS_ROWS, per column for
 * FFT2D_PASS_COLS) -> complex64.  Device buffers, asynchronous. */
FFT2D_API fft2d_status fft2d_h16_unpack(int rows, int cols, const void *in, const int *exps,
                                        int axis, void *out, void *stream);

/*
 * Gaussian low-pass multiply of an unshifted 2D spectrum in place (the
 * filter step of FFT -> filter -> inverse FFT, the image-filtering use that
 * motivates the paper, Section 1):
 *   X[k][l] *= exp(-d_k^2/(2 sigma_rows^2)) * exp(-d_l^2/(2 sigma_cols^2)),
 *   d_k = min(k, rows-k), d_l = min(l, cols-l) (frequency distance in bins).
 * dtype FFT2D_C64 (complex64) or FFT2D_C32H (half2; the factor is <= 1, so
 * per-line exponents stay valid).  Device buffer, asynchronous.
 */
FFT2D_API fft2d_status fft2d_lowpass(int rows, int cols, int dtype, void *data, float sigma_rows,
                                     float sigma_cols, void *stream);

/* ------------------------------------------------------------------ serving
 * A continuous-batching request loop on the current device.  Clients submit
 * requests on host buffers (pin them for full copy speed).  A scheduler
 * thread admits queued requests in arrival order while the device memory
 * they need (complex64: 8 B/pixel; half2: 4 B/pixel + 2 rows + cols
 * exponents) fits the HBM budget, launches everything admitted so far as one
 * batch on an idle stream (copies in, grouped FFT launches for both storage
 * types, low-pass, inverse, copies out), keeps up to `streams` batches in
 * flight so new arrivals overlap running work, and recycles device buffers
 * through a resident pool.  Plans stay resident.  Results do not depend on
 * what else is in flight: every kernel computes the same bits alone and in a
 * batch.  Half2 requests cross the host link as half2 (4 B/pixel each way).
 */
#define FFT2D_OP_FORWARD 0   /* forward 2D FFT */
#define FFT2D_OP_LOWPASS 1   /* forward FFT, Gaussian low-pass (sigma = side/8), inverse FFT */

#define FFT2D_SERVE_SIMULATE 1   /* flags: no CUDA calls, modelled device time (testing) */

typedef struct fft2d_server_s *fft2d_server_t;

typedef struct {
    int op;           /* FFT2D_OP_FORWARD or FFT2D_OP_LOWPASS */
    int rows, cols;   /* powers of two, <= FFT2D_MAX_SIDE */
    int dtype;        /* storage: FFT2D_C64 or FFT2D_C32H (sides >= 2) */
    const void *in;   /* host input: rows*cols complex64, or rows*cols half2 (FFT2D_C32H) */
    void *out;        /* host result in the same storage (may equal in) */
    const int *in_exp;  /* FFT2D_C32H: host, rows exponents of the input, one per row
                           (the format of fft2d_h16_pack); NULL for complex64 */
    int *out_exp;       /* FFT2D_C32H: host, receives cols exponents of the result, one
                           per column (the format fft2d_exec_h16 writes); NULL for complex64 */
} fft2d_request;

typedef struct {
    long long submitted, completed, rejected, queued, batches, peak_device_bytes;
    double mean_batch_size;
    double p50_ms, p99_ms, mean_ms, max_ms;   /* submit -> result on the host */
    double throughput_rps;                    /* completed / (last completion - first submit) */
} fft2d_serve_stats;

/* Create a server with an HBM budget (bytes of device buffers it may hold)
 * and 1..16 streams.  flags: 0 or FFT2D_SERVE_SIMULATE. */
FFT2D_API fft2d_status fft2d_serve_create(size_t hbm_budget_bytes, int streams, int flags,
                                          fft2d_server_t *out);

/* Queue one request; *ticket identifies it.  A request whose buffers alone
 * exceed the budget is refused with FFT2D_ERR_BUDGET.  Non-blocking. */
FFT2D_API fft2d_status fft2d_serve_submit(fft2d_server_t srv, const fft2d_request *req,
                                          unsigned long long *ticket);

/* Wait up to timeout_ms (< 0: forever) for a ticket; returns its status (or
 * FFT2D_ERR_TIMEOUT if still running) and its latency in ms.  Each ticket
 * can be waited for once. */
FFT2D_API fft2d_status fft2d_serve_wait(fft2d_server_t srv, unsigned long long ticket,
                                        int timeout_ms, double *latency_ms);

/* Counters and latency percentiles of all completed requests. */
FFT2D_API fft2d_status fft2d_serve_stats_get(fft2d_server_t srv, fft2d_serve_stats *out);

/* Finish all queued work, then release the server. */
FFT2D_API fft2d_status fft2d_serve_destroy(fft2d_server_t srv);

/*
 * Host-only: write the rotation-factor table that a plan uploads for an axis
 * of 2^L points (0 <= L <= 14) into out[0 .. 2*(2^L - 1)), as (re, im) float
 * pairs.  Stage s (1..L) occupies entries [2^(s-1) - 1, 2^s - 1) and entry
 * 2^(s-1) - 1 + j holds W_{2^s}^j = exp(-+2*pi*i*j/2^s) (minus sign for
 * FFT2D_FORWARD), computed in FP64 with exact quarter-turn values and rounded
 * to FP32 -- the paper's per-stage "secondary texture" (Section 3.1), one row
 * per stage, compacted to the entries a stage uses.  Needs no GPU.
 */
FFT2D_API fft2d_status fft2d_stage_table(int L, int dir, float *out);

/* Largest side accepted by fft2d_exec_noalloc. */
#define FFT2D_NOALLOC_MAX_SIDE 4096

/*
 * The whole 2D transform (as fft2d_exec) without any device allocation, for
 * callers that cannot allocate: a plug-in inside a host application that
 * manages every byte of the device itself (a cudaMalloc behind its back
 * breaks its accounting or fails because it reserved the whole device), code
 * in a process whose caching allocator already holds the free memory, and
 * latency-bound paths where cudaMalloc's implicit device synchronisation is
 * not allowed.  The paper has no counterpart; this is a deployment
 * convenience.
 *
 * rows, cols: powers of two, 1 <= side <= FFT2D_NOALLOC_MAX_SIDE (4096);
 * larger sides return FFT2D_ERR_TOO_LARGE (use a plan for them).  dir is
 * FFT2D_FORWARD or FFT2D_INVERSE; in/out are caller-owned device buffers of
 * rows*cols complex64 pixels (in == out allowed).  Asynchronous on `stream`.
 *
 * Instead of a plan, the rotation-factor tables and the kernels' status word
 * live in one static device array of about 64 KB that every device holds from
 * the library's load until the process exits.  Each call rewrites the tables
 * for its shape and direction and clears the status word on the stream, so
 * calls that overlap on the GPU (different streams, or different threads on
 * one device) race on that array: serialise them.  The first call on each
 * device looks up the array's device address (cudaGetSymbolAddress); make
 * that first call before any stream capture.  It calls no cudaMalloc or
 * cudaFree.  A bounded device wait that gives up is not reported here (use a
 * plan and fft2d_sync_status for that).
 */
FFT2D_API fft2d_status fft2d_exec_noalloc(int rows, int cols, int dir, const void *in, void *out,
                                          void *stream);

/*
 * Batch autotuner: for every group of fft2d_exec_batched's grouped launches
 * in this batch (pass, axis length, direction), time each grouped-kernel
 * variant (rows: plain, 32 values per thread; columns: plain, half-width
 * tiles, persistent TMA-fed with TMA stores, with per-thread stores, or with
 * half of each) and keep the fastest per (pass, axis length) in
 * the process-wide tuning table (and FFT2D_TUNE_CACHE).  Later
 * fft2d_exec_batched calls use the winners.  The buffers are overwritten
 * with intermediate results (the passes run several times).  Synchronous.
 */
FFT2D_API fft2d_status fft2d_autotune_batched(int n, const fft2d_plan_t *plans,
                                              const void *const *in, void *const *out,
                                              void *stream);

/* Grouped-kernel variants of fft2d_exec_batched: how many a pass has, the
 * name of variant `index` ("" when out of range), the variant the calling
 * thread's current device uses for a pass over lines of 2^L points (-1 on a
 * bad argument or no device), and forcing one (-1: back to the default).  A
 * forced choice goes into the same process-wide table as a tuned winner.  A
 * variant that cannot serve a group (e.g. the TMA column kernel on an image
 * whose width is not a whole number of tiles) falls back to "plain". */
FFT2D_API int fft2d_batch_variant_count(int pass);
FFT2D_API const char *fft2d_batch_variant_name(int pass, int index);
FFT2D_API int fft2d_batch_get_variant(int pass, int L);
FFT2D_API fft2d_status fft2d_batch_set_variant(int pass, int L, int variant);

/* Static text for a status code. */
FFT2D_API const char *fft2d_strerror(int status);

/* Text of the calling thread's last CUDA failure ("" if none). */
FFT2D_API const char *fft2d_last_error(void);

/* ABI version (major * 100 + minor). */
FFT2D_API int fft2d_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FFT2D_H */

/*
 * mxgemm -- mixed-datatype general matrix multiplication on one GB300 GPU.
 *
 *     C := beta * C + alpha * op(A) * op(B)
 *
 * following Van Zee, Parikh and van de Geijn, "Supporting mixed-datatype matrix
 * multiplication within the BLIS framework" (arXiv 1901.06015). Each of A, B and C
 * is stored independently as single or double precision, real or complex; the
 * computation precision is chosen separately (4 x 4 x 4 storage datatypes x 2
 * computation precisions = 128 combinations).
 *
 * Semantics (the same for every entry point below):
 *  - Domains (Sec. 4.2, Fig. "mixeddom"): real operands behave as complex with zero
 *    imaginary part, the product P = op(A) op(B) is formed, and
 *        C real:    C := Re(beta) C + Re(alpha) Re(P)
 *        C complex: C := beta C + alpha P
 *    so with C real the imaginary parts that cannot reach C are never computed on
 *    (cases 1a, 1b, 2ab), and with A and B real only Re(C) receives the product
 *    while Im(C) is only scaled by beta (case 1c).
 *  - Precision (Sec. 5.1): A and B are cast to the computation precision (their
 *    "target datatype": own domain, computation precision) and the whole length-k
 *    sum is accumulated in it; the result is cast to C's storage precision when it
 *    is accumulated into C (Sec. 5.1.3, Sec. 6.3).
 *  - Scalars (Sec. 7.1, option 1 for both): alpha is cast to the computation
 *    precision, beta to C's storage precision, and alpha*AB is cast to C's precision
 *    before beta*C is added in C's precision. Sec. 7.2: complex beta is projected when
 *    C is real; complex alpha is projected in case 0, honoured in case 3, and a
 *    non-zero Im(alpha) is rejected (MXG_ECOMPLEX_ALPHA) in cases 1a, 1b, 1c, 2ab,
 *    2ac, 2bc. Rounding is round-to-nearest-even.
 *  - beta == 0: C is not read (NaN in C does not propagate). alpha == 0 (after the
 *    cast to the computation precision) or k == 0: A and B are not read and
 *    C := beta C. m == 0 or n == 0: nothing happens.
 *
 * Storage (Sec. 2.2.1, Sec. 3 Fig. "hypoapi"): element (i, j) of a stored matrix X
 * lives at X + (i * rs + j * cs) elements of X's datatype; a complex element is one
 * unit (real part first, then imaginary). Strides are in elements, >= 1 for every
 * dimension longer than 1: column-major (rs = 1), row-major (cs = 1) and general
 * storage are all accepted for each operand independently. op(A) is m x k; A is
 * stored k x m when transa is MXG_TRANS or MXG_CONJTRANS (induced transposition,
 * Sec. 2.2.2). MXG_CONJ conjugates without transposing (Sec. 2.2.3). C must not
 * overlap itself; A and B may alias each other but not C.
 *
 * Ownership and ordering: the caller owns A, B and C (device memory). Work is
 * enqueued on the handle's stream and is asynchronous; no pointer is kept after the
 * call's work has passed on that stream. Errors are returned as status codes; no
 * entry point aborts or throws.
 */
#ifndef MXGEMM_H
#define MXGEMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Storage datatypes (Sec. 3: domain x precision). Beyond the paper's four, the
 * 16-bit precisions of Sec. 5.3: MXG_H real binary16, MXG_K complex binary16, MXG_B
 * real bfloat16, MXG_W complex bfloat16 (a complex element is (re, im), 4 bytes). */
enum { MXG_S = 0, MXG_D = 1, MXG_C = 2, MXG_Z = 3, MXG_H = 4, MXG_K = 5, MXG_B = 6, MXG_W = 7 };

/* Transposition values (Sec. 3, incl. conjugation without transposition). */
enum { MXG_NOTRANS = 0, MXG_TRANS = 1, MXG_CONJ = 2, MXG_CONJTRANS = 3 };

/* Computation precision (Sec. 5.1.1). MXG_PREC_OF_C: that of C's storage.
 * MXG_PREC_H / MXG_PREC_B (Sec. 5.3): A and B are rounded to binary16 / bfloat16 and
 * the products are summed in FP32 on the tensor cores (method MXG_METHOD_TC16); alpha
 * is rounded to that precision. */
enum { MXG_PREC_S = 0, MXG_PREC_D = 1, MXG_PREC_OF_C = 2, MXG_PREC_H = 3, MXG_PREC_B = 4 };

/* Contraction methods. FFMA: plain FP32 fused multiply-add (single);
 * TF32X3 / BF16X3: split-precision tensor-core products hi*hi + hi*lo + lo*hi with
 * FP32 accumulation (single); DMMA: FP64 tensor-core mma (double); DFMA: plain FP64
 * fused multiply-add (double); TC16: one tensor-core pass on binary16 / bfloat16
 * operands with FP32 accumulation (computation precision h / b). AUTO picks FFMA for
 * single, DFMA for double and TC16 for the 16-bit precisions. */
enum {
  MXG_METHOD_AUTO = 0,
  MXG_METHOD_FFMA = 1,
  MXG_METHOD_TF32X3 = 2,
  MXG_METHOD_BF16X3 = 3,
  MXG_METHOD_DMMA = 4,
  MXG_METHOD_DFMA = 5,
  MXG_METHOD_TC16 = 6
};

/* Status codes. */
enum {
  MXG_OK = 0,
  MXG_EINVAL = 1,          /* bad enum, negative size, null pointer with work to do,
                              stride < 1 on a dimension longer than 1, C overlapping
                              itself, method not of the computation precision */
  MXG_ECOMPLEX_ALPHA = 2,  /* Im(alpha) != 0 in case 1a, 1b, 1c, 2ab, 2ac or 2bc (Sec. 7.2) */
  MXG_ENOMEM = 3,          /* workspace allocation failed or caller workspace too small */
  MXG_ECUDA = 4,           /* a CUDA runtime call failed (see mxg_last_cuda_error) */
  MXG_ETIMEOUT = 5,        /* a device-side wait ran out of its iteration limit */
  MXG_ENOTSUP = 6,         /* method not available on this device */
  MXG_ESCRATCH = 7,        /* mxgemm_noalloc: the call needs more scratch than the fixed
                              MXG_NOALLOC_SCRATCH_BYTES buffer holds */
  MXG_EACCURACY = 8        /* the split-precision method cannot keep the normwise error
                              within 4 k u_s at this k (see MXG_SPLIT_MIN_K_*) */
};

/* Smallest k at which a split-precision method is accepted. Its products drop terms of
 * relative size up to 3 u_p^2 (u_p the unit roundoff of the plane format: 2^-8 for
 * BF16, 2^-11 for TF32), a floor independent of k. The stated accuracy is a normwise
 * error of at most 4 k u_s (u_s = 2^-24), so below some k the floor alone can exceed
 * it. The limits leave room for the floor (774 u_s for BF16X3, 12 u_s for TF32X3),
 * the FP32 accumulation on the tensor cores (taken as at most 4 u_s per MMA step on
 * the sum of magnitudes, 3 K'/16 resp. 3 K'/8 steps with K' <= 2k) and the epilogue's
 * roundings (about 5.5 u_s): BF16X3 needs 2.5 k >= 780, TF32X3 k >= 18. A call below
 * the limit returns MXG_EACCURACY and enqueues nothing; FFMA and TF32X3 cover it. */
#define MXG_SPLIT_MIN_K_BF16X3 320
#define MXG_SPLIT_MIN_K_TF32X3 32

/* Domain cases of Fig. "mixeddom", as returned in mxg_plan_info.domain_case:
 * index = 4*[C complex] + 2*[A complex] + [B complex]. */
enum {
  MXG_CASE_0 = 0, MXG_CASE_1B = 1, MXG_CASE_1A = 2, MXG_CASE_2AB = 3,
  MXG_CASE_1C = 4, MXG_CASE_2BC = 5, MXG_CASE_2AC = 6, MXG_CASE_3 = 7
};

typedef struct mxg_context* mxg_handle;

/* Description of the real gemm a call reduces to (host-side planning only). */
typedef struct {
  int domain_case;          /* MXG_CASE_* (Fig. "mixeddom") */
  int comp_prec;            /* resolved computation precision: MXG_PREC_S, _D, _H or _B */
  int method;               /* resolved MXG_METHOD_* */
  int whole_op_transposed;  /* 1 if computed as C^T := op(B)^T op(A)^T (Sec. 2.2.5) */
  int64_t Mr, Nr, Kr;       /* dimensions of the real product (M', N', K') */
  int real_products;        /* R = M'N'K' / (mnk): 1, 2 or 4 (flops = 2mnk R) */
  double flops;             /* useful flops 2*m*n*k*R (Fig. "mixeddom") */
  size_t workspace_bytes;   /* device workspace the call needs (packed operands, split-K sums) */
  int k_splits;             /* split-K slices (1: none; see mxg_set_split_k) */
} mxg_plan_info;

/*
 * mxgemm: the mixed-datatype gemm of Sec. 3 Fig. "hypoapi", with domain and
 * precision folded into one datatype code per operand (dtX in MXG_S..MXG_Z) and the
 * computation precision precAB as comp_prec. Runs on the calling thread's current
 * device, on the default (legacy) stream, with a library-owned workspace that grows
 * as needed. Pointers are device pointers. Returns MXG_OK or an error status; on an
 * error nothing is enqueued and C is unchanged.
 */
int mxgemm(int transa, int transb, int64_t m, int64_t n, int64_t k,
           double alpha_re, double alpha_im,
           const void* A, int dtA, int64_t rsA, int64_t csA,
           const void* B, int dtB, int64_t rsB, int64_t csB,
           double beta_re, double beta_im,
           void* C, int dtC, int64_t rsC, int64_t csC,
           int comp_prec);

/*
 * mxgemm_ex: as mxgemm, on handle h (its device, stream and workspace) with an
 * explicit contraction method (MXG_METHOD_*). A method of the other precision than
 * the resolved computation precision is MXG_EINVAL.
 */
int mxgemm_ex(mxg_handle h, int method, int transa, int transb,
              int64_t m, int64_t n, int64_t k,
              double alpha_re, double alpha_im,
              const void* A, int dtA, int64_t rsA, int64_t csA,
              const void* B, int dtB, int64_t rsB, int64_t csB,
              double beta_re, double beta_im,
              void* C, int dtC, int64_t rsC, int64_t csC,
              int comp_prec);

/*
 * mxg_plan: validate a call and describe the real gemm it reduces to (domain case,
 * M', N', K', R, method, workspace). Host only: makes no CUDA call, so it works
 * without a GPU. Pointers may be NULL here (they are not dereferenced or checked).
 * Returns the status mxgemm_ex would return for a validation failure, else MXG_OK.
 */
int mxg_plan(int method, int transa, int transb, int64_t m, int64_t n, int64_t k,
             double alpha_re, double alpha_im,
             int dtA, int64_t rsA, int64_t csA,
             int dtB, int64_t rsB, int64_t csB,
             int dtC, int64_t rsC, int64_t csC,
             int comp_prec, mxg_plan_info* info);

/* Handles. mxg_create binds the handle to the calling thread's current device and
 * to the default stream. mxg_destroy frees the library-owned workspace (after
 * synchronising the handle's stream). */
int mxg_create(mxg_handle* h);
int mxg_destroy(mxg_handle h);

/* Literal complex alpha on h (off by default). Sec. 7.2 rejects a non-zero Im(alpha) in
 * cases 1a, 1b, 1c, 2ab, 2ac and 2bc and names the alternative, a literal
 * interpretation in which all five operands' domains are taken at face value. With
 * on != 0, calls on h take that reading: C := beta*C + alpha*op(A)*op(B) in complex
 * arithmetic, projected onto C's domain (C real: C := Re(beta) C + Re(alpha AB)).
 * With C real, alpha is folded into the pack of the complex operand (the "special
 * packing function" for Re(alpha A) of the paper's footnote); with C complex the
 * epilogue applies the complex alpha. Grouped launches and the server keep the
 * paper's rule. */
int mxg_set_literal_alpha(mxg_handle h, int on);

/* Split-K on h (off by default): the paper's C_temp in the computation precision
 * (Secs. 6.2-6.4) used for parallelism over K. K' is cut into slices computed by
 * separate CTAs into a workspace of partial sums (splits x M' x N' in the computation
 * precision); a reduction adds the slices in a fixed order and applies the epilogue
 * once, so results are deterministic but round differently from the unsplit call.
 * mode: 0 off; 1 automatic (split only when the tile grid has fewer tiles than the
 * device has SMs, keeping at least 512 k per slice); n >= 2 exactly n slices (fewer
 * when K' is short). Applies to the FFMA, DFMA and DMMA methods; the split-precision
 * tensor-core methods and grouped launches do not split. */
int mxg_set_split_k(mxg_handle h, int mode);

/* CTA pairs for the tensor-core methods (TF32X3, BF16X3, TC16) on h: mode 0 automatic
 * (= pairs), 1 pairs, 2 one CTA per tile. A pair is a cluster of two CTAs on two SMs
 * computing a 256 x 256 tile with tcgen05 cta_group::2 MMAs; each CTA loads its own
 * half of the tile's A and B rows (128-byte k rows), so the operands cost a third fewer
 * bytes, and half the requests, from L2 per flop than single-CTA 128 x 256 tiles. With
 * the stream-K tail off (mxg_set_stream_k mode 0) the two kernels give the same results
 * bit for bit (tested; same products, accumulated in the same order along k). */
int mxg_set_cta_pairs(mxg_handle h, int mode);

/* Stream-K tail of the CTA-pair kernel on h: mode 0 off, 1 automatic (the default), 2
 * whenever the last wave of pair tiles is partial. With T pair tiles on P resident pairs
 * and r = T mod P > 0, the last r tiles are cut along k into P equal ranges, one per
 * pair, so no pair idles through a partial last wave. Each range's FP32 partial
 * accumulator goes to the workspace; the range that finishes a tile last adds the
 * tile's partials in increasing k and applies the epilogue (Sec. 7.1) to the sum, so
 * the result is the same from run to run. It differs from a whole-tile run only in the
 * FP32 summation order along k; the stated bound holds for both. Automatic mode runs
 * the tail when the pairs left idle by the last wave are at least 6% of the whole run
 * and each range has at least 16 k blocks. The tail adds (SMs / 2) x 512 KB (+
 * counters) to the workspace; a caller workspace that holds the rest of the plan but
 * not this runs without the tail.
 * mxgemm_noalloc and the server never use it. */
int mxg_set_stream_k(mxg_handle h, int mode);

/* Stream for subsequent calls on h (a cudaStream_t; NULL = legacy default stream). */
int mxg_set_stream(mxg_handle h, void* stream);

/* Caller-owned device workspace for subsequent calls on h: ptr must be 256-byte
 * aligned; a call whose plan needs more than bytes returns MXG_ENOMEM. ptr = NULL
 * returns to the library-owned, growing workspace. The caller keeps ownership and
 * must not reuse the memory until work enqueued on h has completed. */
int mxg_set_workspace(mxg_handle h, void* ptr, size_t bytes);

/* Device error word of h: nonzero if something went wrong on the device since the last
 * call to this function (which clears it): bit 0 (1) a device-side wait ran out of its
 * iteration limit; bit 1 (2), debug builds only (mxg_debug_bounds), a pack kernel or an
 * epilogue computed an element address outside the extent its arguments describe and
 * skipped that access. Synchronises h's stream. Returns MXG_OK or MXG_ECUDA; *flag
 * receives the word. */
int mxg_check_device_error(mxg_handle h, int* flag);

/*
 * Grouped persistent launch: many independent gemms of uneven shapes and mixed
 * datatype combinations in few launches. Each problem has the semantics of mxgemm
 * (all of the rules above); problems must not write overlapping C. The paper's
 * argument (Sec. 2.2.4) that datatype handling is orthogonal to how the loops are
 * parallelised is what lets problems of different datatypes share one launch.
 *
 * mxg_group_create validates and plans every problem (the first invalid one makes it
 * fail with that problem's status; *first_bad receives its index when first_bad is not
 * NULL), buckets the problems by computation precision and method, and builds on the
 * device: the packed operands of every problem, one pack work list per bucket and one
 * (problem, tile) work list per bucket, ordered longest-first. A run is then one
 * grouped pack launch and one persistent contraction launch per bucket (plus a
 * C := beta*C launch per problem with k == 0 or alpha == 0).
 *   method_s: MXG_METHOD_AUTO or MXG_METHOD_FFMA (single precision on the FP32 pipe), or
 *             MXG_METHOD_TF32X3 / MXG_METHOD_BF16X3 (single precision on the tensor
 *             cores; problems below the method's smallest k, MXG_SPLIT_MIN_K_*, run in
 *             the FFMA bucket instead);
 *   method_d: MXG_METHOD_AUTO (= DFMA), MXG_METHOD_DMMA or MXG_METHOD_DFMA (double bucket);
 *   the 16-bit computation precisions run in two tensor-core buckets (TC16, binary16 and
 *   bfloat16). Tensor-core buckets use each problem's own tensor maps, encoded at create
 *   time, on a persistent 128 x 256-tile tcgen05 kernel; their bounded waits report a
 *   timeout through the handle's error word (mxg_check_device_error);
 *   flags:    MXG_GROUP_TUNE  -- time each bucket's candidate kernels and schedules
 *                                 (into scratch copies of C, so the problems' C are not
 *                                 touched) and keep the fastest; decisions are cached in
 *                                 the process by a signature of the bucket;
 *             MXG_GROUP_GRAPH -- capture the run in a CUDA graph, replayed by each
 *                                 mxg_group_run.
 * The group owns its device memory (one allocation) until mxg_group_destroy, which
 * synchronises h's stream. The problems' A, B and C pointers are read at create time
 * and used by every run; their contents are read and written at run time.
 */
typedef struct {
  int transa, transb;
  int64_t m, n, k;
  double alpha_re, alpha_im, beta_re, beta_im;
  const void* A; int dtA; int64_t rsA, csA;
  const void* B; int dtB; int64_t rsB, csB;
  void* C; int dtC; int64_t rsC, csC;
  int comp_prec;
} mxg_problem;

typedef struct mxg_group_s* mxg_group;

enum { MXG_GROUP_TUNE = 1, MXG_GROUP_GRAPH = 2 };

int mxg_group_create(mxg_handle h, int64_t count, const mxg_problem* probs, int method_s, int method_d,
                     int flags, mxg_group* out, int64_t* first_bad);
/* Enqueue one run of the group on its handle's stream (asynchronous). */
int mxg_group_run(mxg_group g);
/* Write a one-line JSON description (buckets, kernels, schedules, tiles, tuned times)
 * into buf (NUL-terminated, truncated to len). */
int mxg_group_describe(mxg_group g, char* buf, size_t len);
int mxg_group_destroy(mxg_group g);

/* One-shot grouped call: create (no tuning, no graph), run, synchronise, destroy. */
int mxgemm_grouped(mxg_handle h, int64_t count, const mxg_problem* probs);

/* Save / load the autotuner's decisions (text, one line per bucket signature). */
int mxg_tune_save(const char* path);
int mxg_tune_load(const char* path);

/*
 * Serving loop: a request server with continuous batching. Requests (each an
 * mxg_problem with the semantics of mxgemm, device operands owned by the caller) are
 * submitted from any host thread at any time. A worker thread admits them by HBM
 * footprint -- bytes of A, B, C plus the packed operands -- while the footprint of the
 * requests in flight stays within hbm_budget_bytes; their packed operands are carved
 * from one device arena of that size (first-fit free list with coalescing) and stay
 * resident until the request completes. Admitted work is spread over n_streams
 * streams and overlaps on the device: requests of at most small_flops useful flops go
 * to a high-priority stream, larger ones round-robin over the others (flag
 * MXG_SERVE_FIFO instead sends every request to stream 0 in submission order, with no
 * priority, which is the serial baseline). Small requests are batched: those admitted
 * while the previous wave still runs on the high-priority stream wait for it to finish
 * and then run together as one wave -- one grouped pack launch and one persistent
 * grouped contraction per computation precision over all of their tiles (the kernels of
 * mxg_group_run, so each result equals the separate call's bit for bit). Plain
 * FFMA / DFMA / DMMA requests join waves; a request on the split-precision or 16-bit
 * tensor-core methods, or C := beta*C only, runs on its own. When the head of the queue
 * does not fit, later small requests that fit are admitted past it, until the head has
 * waited 50 ms. Completion is observed with one CUDA event per wave or request; times
 * are seconds on the server's clock (mxg_server_now): arrival = when submitted, admit =
 * when its memory was reserved, done = when the request's last kernel finished on the
 * device.
 */
typedef struct mxg_server_s* mxg_server;

typedef struct {
  uint64_t id;        /* as returned by mxg_server_submit */
  int status;         /* MXG_OK or the error of planning / launching */
  int stream;         /* stream index the request ran on (-1 if it never ran) */
  double arrival, admit, done;
  double flops;       /* useful flops 2mnk R */
  size_t footprint;   /* bytes counted against the budget */
} mxg_completion;

typedef struct {
  uint64_t submitted, admitted, completed, failed;
  size_t bytes_in_flight, peak_bytes_in_flight, budget;
  int64_t max_in_flight, queue_len;
  uint64_t waves, wave_requests;   /* grouped launches of small requests, and the requests they held */
} mxg_server_stats;

enum { MXG_SERVE_FIFO = 1 };

int mxg_server_create(int n_streams, size_t hbm_budget_bytes, double small_flops, int method_s, int method_d,
                      int flags, mxg_server* out);
/* Thread-safe; never blocks on the device. *id receives the request id. */
int mxg_server_submit(mxg_server s, const mxg_problem* p, uint64_t* id);
/* Move up to max completions into out (*n receives the count); never blocks. */
int mxg_server_poll(mxg_server s, mxg_completion* out, int max, int* n);
/* Block until every submitted request has completed (or timeout_s passes: MXG_ETIMEOUT). */
int mxg_server_drain(mxg_server s, double timeout_s);
int mxg_server_get_stats(mxg_server s, mxg_server_stats* st);
/* Device error word of s (shared by its streams): nonzero if a device-side wait in a
 * served request ran out of its limit since the last call to this function (which
 * clears it). Waits for the work in flight on s's streams. Returns MXG_OK or
 * MXG_ECUDA; *flag receives the word. */
int mxg_server_check_device_error(mxg_server s, int* flag);
double mxg_server_now(mxg_server s);
/* Drains, stops the worker, frees the arena and streams. */
int mxg_server_destroy(mxg_server s);

/* Phase timing on h (tracing). When on, every call on h records CUDA events on h's
 * stream before its pack launches, between the packs and the contraction launch, and
 * after the contraction. mxg_phase_times synchronises h's stream, returns the summed
 * milliseconds of the pack phase and of the contraction phase (the contraction kernel
 * with its fused epilogue) and the number of contraction launches recorded since the
 * last query, then forgets them. Turning timing off also forgets them. */
int mxg_set_phase_timing(mxg_handle h, int on);
int mxg_phase_times(mxg_handle h, double* pack_ms, double* contraction_ms, int64_t* launches);

/*
 * mxgemm_noalloc: mxgemm_ex without any device allocation. (The paper has no
 * counterpart; this entry point exists for callers that cannot call cudaMalloc:
 * latency-critical loops that cannot take the implicit device synchronisation of
 * cudaMalloc/cudaFree, and applications whose device memory is all owned by another
 * allocator -- a framework's caching pool or a fixed memory plan -- that forbids side
 * allocations.)
 *
 * Same arguments and semantics as mxgemm_ex, with a cudaStream_t (NULL = legacy
 * default stream) in place of the handle. The packed operands live in one fixed
 * file-scope device array of MXG_NOALLOC_SCRATCH_BYTES bytes, which every GPU that
 * loads this code holds until the process exits; the call makes no cudaMalloc,
 * cudaFree or other allocating call. A problem whose packed operands need more than
 * that (see mxg_plan's workspace_bytes) is rejected with MXG_ESCRATCH and nothing is
 * enqueued. The first call on a device (or the first mxgemm_noalloc_check_device_error
 * there) looks up the array's device address, once per device, with that device
 * current. All calls in the process share the one array and it keeps the last call's
 * contents (every call rewrites all of the part it uses, so nothing needs clearing),
 * so calls whose work may overlap on the GPU -- on different streams, or from several
 * host threads -- race on it: serialise them on one stream.
 *
 * Timeouts: the tensor-core methods (TF32X3, BF16X3, TC16) bound every device-side
 * wait; a wait that runs out makes the kernel skip its stores and set this entry
 * point's own device error word (a second file-scope device int, shared by all calls
 * like the array). The call itself has returned MXG_OK by then, so check the word with
 * mxgemm_noalloc_check_device_error after the work.
 */
#define MXG_NOALLOC_SCRATCH_BYTES (32u << 20)
int mxgemm_noalloc(void* stream, int method, int transa, int transb,
                   int64_t m, int64_t n, int64_t k,
                   double alpha_re, double alpha_im,
                   const void* A, int dtA, int64_t rsA, int64_t csA,
                   const void* B, int dtB, int64_t rsB, int64_t csB,
                   double beta_re, double beta_im,
                   void* C, int dtC, int64_t rsC, int64_t csC,
                   int comp_prec);

/* The device error word of mxgemm_noalloc on the current device: synchronises
 * `stream` (a cudaStream_t, NULL = legacy default stream), writes the word to *flag
 * (nonzero: a device-side wait of some mxgemm_noalloc call ran out of its limit since
 * the word was last cleared) and clears it. Allocates nothing. Returns MXG_OK or
 * MXG_ECUDA. */
int mxgemm_noalloc_check_device_error(void* stream, int* flag);

/* Self-test of the device-side wait limit: launches one kernel that waits on an
 * mbarrier nothing will ever arrive on, for at most `seconds` (0 < seconds <= 10), on
 * h's stream. Returns MXG_ETIMEOUT when the wait ran out and reported it through the
 * error word (the expected outcome; the word is cleared again), MXG_OK if it did not
 * report, or an error status. The GPU context stays usable. */
int mxg_selftest_wait_timeout(mxg_handle h, double seconds);

/* Human-readable text of a status code (static storage). */
const char* mxg_strerror(int status);

/* The last CUDA runtime error code seen by the library on this thread (0 if none). */
int mxg_last_cuda_error(void);

/* Library version as major*10000 + minor*100 + patch. */
int mxg_version(void);

/* 1 if this library is the debug build with device-side bounds checks of every pack and
 * epilogue access (compiled with MXG_DEBUG_BOUNDS; violations set bit 1 of the device
 * error word instead of touching memory), else 0. */
int mxg_debug_bounds(void);

#ifdef __cplusplus
}
#endif

#endif /* MXGEMM_H */

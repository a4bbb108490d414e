/*
 * truncmul.h - C ABI of a GB300 (sm_103a) library for full, low and high
 * products of n-bit integers, after D. Harvey, "Faster truncated integer
 * multiplication".
 *
 * Definitions (Section 1 of the paper). For integers 0 <= u, v < 2^n:
 *   full product  uv, a 2n-bit integer;
 *   low product   the unique 0 <= w < 2^n with w == uv (mod 2^n);
 *   high product  any 0 <= w <= 2^n with |uv - 2^n w| < 2^n (at most two
 *                 values qualify; w = 2^n is possible).
 *
 * Method. Full products follow Algorithm 1 (split into b-bit digits, one real
 * cyclic convolution of length >= 2N - 1, round, overlap-add). Low products
 * follow Algorithm 2 (Section 3): digits -> alpha* map -> real cyclic
 * convolution of length N -> beta* map -> round(2^b W_i) -> overlap-add mod
 * 2^n. High products follow Algorithm 3 (Section 4): digits of u 2^((N+1)b-n)
 * -> gamma-dagger -> convolution plus the auxiliary scalar theta -> delta-dagger
 * -> round -> round(t). Every step runs in CUDA kernels of this library; the
 * convolution is an FP64 real FFT. The parameters (b, N, lambda) come from a
 * worst-case FP64 error bound, so that every rounded coefficient is exact; each
 * call measures the largest distance of a rounded value to its integer (the
 * "margin") and fails with TM_EPRECISION if it exceeds the bound.
 *
 * Limb layout. Every integer is a little-endian array of uint64_t limbs (limb
 * 0 holds bits 0..63). u and v have ceil(n/64) limbs each; bits at positions
 * >= n of their top limb must be zero (they are ignored). Outputs:
 *   full: 2*ceil(n/64) limbs;
 *   low:  ceil(n/64) limbs, bits >= n cleared;
 *   high: floor(n/64) + 1 limbs (room for w = 2^n).
 *
 * Memory and ownership. Unless a function says otherwise, u, v and out are
 * DEVICE pointers owned by the caller; out must not overlap u or v (u == v is
 * allowed and squares: one forward map and one forward FFT instead of two). The library owns a plan cache (twiddle and map tables, kept
 * resident per (kind, n) and device) and a workspace per (device, stream),
 * both grown on demand and kept until tm_release() or process exit. Calls on
 * the same stream are ordered; calls on different streams use different
 * workspaces and may run concurrently. The library is thread-safe.
 *
 * Streams and status. `stream` is a cudaStream_t (NULL = the legacy default
 * stream); the device is the current device of the calling thread. Work is
 * enqueued on `stream`; where one operand's FFT passes fill the GPU on their own
 * (tm_report.fwd_streams = 2), v's forward transform runs on a second stream of
 * the workspace, forked from and joined back into `stream` by events, so the call
 * stays ordered on `stream`. If `rep` is NULL the call returns as soon as the work
 * is enqueued and the device-side status (margin check) is collected later
 * by tm_stream_status(). If `rep` is non-NULL the call waits for the stream,
 * fills *rep and returns the device-side status as well.
 */
#ifndef TRUNCMUL_H
#define TRUNCMUL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes (0 = success) ---- */
#define TM_OK          0
#define TM_UNCERTIFIED 1   /* success of tm_mul_params with a (b, N) whose
                              worst-case bound is at or above 1/2: every rounding
                              distance stayed within the caller's limit, but the
                              result is not certified                            */
#define TM_EINVAL     -1   /* bad argument: n = 0, NULL pointer, unknown kind    */
#define TM_ENOMEM     -2   /* device or host allocation failed                   */
#define TM_EPRECISION -3   /* margin above the a-priori bound, or 2^b not
                              dividing c_0: the output must not be trusted       */
#define TM_ETIMEOUT   -4   /* a single-launch product's grid-wide wait gave up
                              after about a second (see tm_set_fused); the
                              output must not be trusted                        */
#define TM_ECUDA      -5   /* a CUDA runtime call failed                         */
#define TM_ERANGE     -6   /* n too large for any FP64 plan of this library      */
#define TM_EALIAS     -7   /* out overlaps u or v                                */

/* Fault injection for callers' tests. With the environment variable
 * TRUNCMUL_FAULT_EMAX_SCALE set to a number in (0, 1] (read once, when the
 * library first enqueues a product), every bound the device checks the margin
 * against is multiplied by it: a small value such as 1e-12 makes every product
 * report TM_EPRECISION through every entry point while computing the same limbs.
 * Other values are ignored.
 * With TRUNCMUL_FAULT_BARRIER=1 (read once), the last CTA of every single-launch
 * product leaves at the first grid barrier without counting itself in, and the first
 * unit of every persistent batch is never reported as finished; the other
 * CTAs' bounded waits (about a second) run out and the call reports TM_ETIMEOUT, the
 * device staying usable. */

/* ---- product kinds ---- */
#define TM_FULL 0          /* Algorithm 1 */
#define TM_LO   1          /* Algorithm 2 */
#define TM_HI   2          /* Algorithm 3 */

/* Largest supported operand size in bits. */
#define TM_MAX_BITS (((uint64_t)1) << 31)

/* Plan and outcome of one call. */
typedef struct tm_report {
  int32_t  kind;      /* TM_FULL, TM_LO or TM_HI                                  */
  int32_t  status;    /* device-side status of the call (TM_OK, TM_EPRECISION, or
                         TM_UNCERTIFIED from tm_mul_params)                       */
  uint32_t b;         /* digit size in bits                                       */
  uint32_t N;         /* real transform length (N of Algorithms 2/3; the cyclic
                         length >= 2 n_digits - 1 of Algorithm 1)                 */
  uint32_t n_digits;  /* digits per operand: N (low), N + 1 (high), ceil((n+1)/b)
                         (full)                                                   */
  uint32_t lam_fwd;   /* terms of alpha* (low) or gamma* (high); 0 for full       */
  uint32_t lam_bwd;   /* terms of beta* (low) or delta* (high); 0 for full        */
  uint32_t fft_passes;/* HBM passes of each complex FFT of length N/2             */
  uint32_t fwd_streams;/* forward FFT launches per pass of a two-operand product
                         in the per-phase sequence: 2 when u's and v's transforms
                         run on two streams (each pass fills the GPU alone), 1 when
                         one launch per pass carries both                         */
  double   margin;    /* largest |2^b Wbar_i - c_i| (low/high) or |W_i - w_i|
                         (full) over the call; filled when rep != NULL           */
  double   e_max;     /* a-priori bound on that distance (< 1/2)                  */
  uint64_t workspace_bytes; /* device workspace the call needs                    */
  uint64_t table_bytes;     /* resident plan tables on the device                 */
} tm_report;

/*
 * tm_mul_full / tm_mul_lo / tm_mul_hi
 *   out  device, see "Limb layout" for the length.
 *   u, v device, ceil(n_bits/64) limbs each.
 *   n_bits in [1, TM_MAX_BITS].
 *   stream cudaStream_t or NULL.
 *   rep  optional (NULL = asynchronous, see above).
 * Returns TM_OK or a negative TM_E* code. On TM_EINVAL/TM_ERANGE/TM_EALIAS
 * nothing is enqueued.
 * Sources: full product - Algorithm 1 and Theorem 2.1; low product -
 * Algorithm 2, Theorem 2.2, Proposition 3.1; high product - Algorithm 3,
 * Theorem 2.3, Proposition 4.1 (the result is the returned round(t), rounding
 * half up, which is one of the at most two admissible values).
 * Execution: products whose complex transform length N/2 is at most 640 run whole
 * in one CTA (one launch); larger ones as the per-phase launch sequence (maps, FFT
 * passes, twist, back map, carry scan). tm_set_fused selects other forms. The
 * results are the same limbs either way.
 */
int tm_mul_full(uint64_t* out, const uint64_t* u, const uint64_t* v, uint64_t n_bits,
                void* stream, tm_report* rep);
int tm_mul_lo(uint64_t* out, const uint64_t* u, const uint64_t* v, uint64_t n_bits,
              void* stream, tm_report* rep);
int tm_mul_hi(uint64_t* out, const uint64_t* u, const uint64_t* v, uint64_t n_bits,
              void* stream, tm_report* rep);

/* The same three operations selected by `kind` (TM_FULL, TM_LO, TM_HI). */
int tm_mul(int kind, uint64_t* out, const uint64_t* u, const uint64_t* v, uint64_t n_bits,
           void* stream, tm_report* rep);

/*
 * tm_mul_params: tm_mul with the caller's digit size b and transform length N,
 * as in the paper's Section 5, where b, N and lambda are chosen by experiment
 * for random operands (its Table 2 lists them).
 *   prm->b      digit size, 4..24.
 *   prm->N      transform length: N of Algorithms 2 and 3, the cyclic length of
 *               Algorithm 1 for the full product; even, 2^a m with m one of
 *               1, 3, 5, 7, 9, 15, 21, 25, 27, 35, 45, 49, 63, 75, 81, 105, 125,
 *               135, 147, 175, 189, at most 2^31; (b, N) must satisfy the
 *               hypotheses of Theorem 2.2 (N b >= n), Theorem 2.3
 *               ((N + 1) b >= n + lg N + 2) or Theorem 2.1 (N >= 2 ceil((n+1)/b) - 1).
 *   prm->limit  the largest rounding distance the call accepts, in [0, 1/2];
 *               0 = e_max when e_max < 1/2, else 3/8.
 * lambda comes from the library's tail budgets for b. rep->e_max is the
 * worst-case bound for (b, N). Below 1/2 the result is certified and the call
 * returns TM_OK. At or above 1/2 (the paper's own setting) the result is NOT
 * certified: the call then returns TM_UNCERTIFIED (a positive code, also in
 * rep->status) in place of TM_OK, and the limit is only a heuristic - a product
 * whose errors reach 1/2 usually also has distances near 1/2, so operands too
 * large for b usually show up as TM_EPRECISION, but nothing guarantees it. With the paper's Table 2 parameters the largest
 * distance on random operands is about 1/4 (n = 10^6, b = 14). Other arguments,
 * layout and errors as tm_mul; TM_EINVAL also for a NULL prm or parameters
 * outside the ranges above.
 */
typedef struct tm_params {
  uint32_t b;
  uint32_t N;
  double limit;
} tm_params;
int tm_mul_params(int kind, uint64_t* out, const uint64_t* u, const uint64_t* v,
                  uint64_t n_bits, const tm_params* prm, void* stream, tm_report* rep);

/*
 * tm_mul_adaptive: tm_mul with a data-dependent digit size. The paper picks b
 * empirically for random inputs (Section 5); the planner's b is the largest the
 * worst-case error bound certifies for ANY operands (all digits at their maximum).
 * This call measures the operands instead: one kernel sums the squares of the
 * balanced digits of u and v for b + 1 at the shortest length that b + 1 admits
 * (the high product's top digits too), the call waits for the stream to read the
 * sums, and the product runs with b + 1 when the same bound with the measured
 * norms ||U||_2 ||V||_2 in place of the worst case stays within the target (and
 * the length is shorter), else with the planner's (b, N). The margin check guards
 * the result as in tm_mul; rep->b, rep->N and rep->e_max (the bound that applied)
 * tell which plan ran. Random operands have norms about sqrt(3) below the worst
 * case. Arguments, layout, errors and results as tm_mul (results are exact either
 * way); the call blocks until the norms are read.
 */
int tm_mul_adaptive(int kind, uint64_t* out, const uint64_t* u, const uint64_t* v,
                    uint64_t n_bits, void* stream, tm_report* rep);

/*
 * tm_mul_host: one product with HOST buffers; waits for `stream` before it
 * returns. u_host == v_host squares.
 * When u_host, v_host and out_host are all page-locked memory mapped into the
 * device's address space (cudaHostAlloc / cudaMallocHost, or cudaHostRegister
 * with mapping, on a 64-bit system) and out_host overlaps neither input, the
 * kernels read the operands and write the product in host memory directly (over
 * NVLink-C2C on a GB300): no staging copies. A page-locked out_host must then be
 * writable from the device (not registered with cudaHostRegisterReadOnly).
 * Otherwise it copies u and v to the device, runs tm_mul on `stream` and copies
 * the result back. On a created stream (not NULL, the legacy or the per-thread
 * default stream) that sequence is recorded once per (stream, kind, n_bits) as a
 * CUDA graph, and later calls re-point its three host copies at the new buffers
 * and launch it (one launch instead of about twenty calls); the recording is
 * redone when the library's buffers for that stream change, and skipped when it
 * cannot be made (pageable host buffers).
 * Limb counts as above. Returns like tm_mul; *rep (optional) is filled.
 */
int tm_mul_host(int kind, uint64_t* out_host, const uint64_t* u_host, const uint64_t* v_host,
                uint64_t n_bits, void* stream, tm_report* rep);

/*
 * tm_mul_events: tm_mul that also records caller-created CUDA events
 * (cudaEvent_t, timing enabled) on `stream` around its phases, for measuring
 * where the device time goes. events[0] is recorded before the first kernel
 * and events[i+1] after phase i, i < TM_NPHASES:
 *   0 digits + forward map (split and convert steps), 1 forward FFTs,
 *   2 real-FFT twist + pointwise product, 3 inverse FFT,
 *   4 back map + rounding (convert back), 5 overlap-add / carry scan.
 * events must hold TM_NPHASES + 1 entries. Same arguments and return values as
 * tm_mul otherwise.
 */
#define TM_NPHASES 6
int tm_mul_events(int kind, uint64_t* out, const uint64_t* u, const uint64_t* v,
                  uint64_t n_bits, void* stream, void* const* events, tm_report* rep);

/*
 * tm_mul_static: tm_mul for callers that cannot allocate device memory, for
 * example code that runs where the memory allocator belongs to someone else, or
 * that must not block on an allocation. The paper has no counterpart; this is
 * a library facility. Everything the call needs on the device (twiddle and map
 * tables, FFT buffers, carry scratch, status word) lives in one file-scope
 * device array of TM_STATIC_SCRATCH_BYTES that every GPU which loads the library
 * holds until the process exits. The call makes no CUDA allocation and no heap
 * allocation; the caller passes u, v and out (device pointers) as for tm_mul.
 *   n_bits must be <= TM_STATIC_MAX_BITS; larger sizes (or a plan that would not
 *   fit the array) return TM_ERANGE and enqueue nothing.
 *   The first call on a device looks the array's device address up
 *   (cudaGetSymbolAddress) with that device current; make that first call
 *   before any stream capture.
 *   Every call on a device shares the same array and leaves its contents for
 *   the next call: each call clears its status word, and rebuilds the plan's
 *   tables unless the previous call on the device used the same plan (kind and
 *   n giving the same digit size and length). Calls that overlap on the GPU - on
 *   different streams, threads or in flight at once - race and must be
 *   serialised by the caller.
 *   Cost of a rebuild: four to six table kernels (twiddles, tangent-form and
 *   twist tables in double-double arithmetic, map rows, and for the high
 *   product kappa and rho^-j, all computed on the device; no host-to-device
 *   copy) before the product's own kernels.
 *   rep as for tm_mul (NULL = asynchronous; a non-NULL rep waits and reports).
 */
#define TM_STATIC_MAX_BITS 65536
#define TM_STATIC_SCRATCH_BYTES (((size_t)4) << 20)
int tm_mul_static(int kind, uint64_t* out, const uint64_t* u, const uint64_t* v,
                  uint64_t n_bits, void* stream, tm_report* rep);

/*
 * Batched products (many products of uneven sizes in one launch).
 *
 * tm_desc describes one product: kind, n_bits and DEVICE pointers as for tm_mul
 * (each out must not overlap its own u or v; different products may share
 * inputs but not outputs).
 *
 * tm_batch_create plans every product, builds the resident tables, allocates the
 * batch's device memory, and records the whole batch as one CUDA graph:
 * products with the same plan (kind, b, N) run as one launch per phase with the
 * product index in the grid, different plans run on concurrent branches of the
 * graph. It waits for `stream` (table set-up) and must not be called while
 * `stream` is being captured. The descriptors are copied; the pointers they
 * hold must stay valid for the life of the batch.
 * tm_batch_launch enqueues the graph on `stream` (one graph launch); the inputs
 * are read when it runs, so a batch can be relaunched on new operand values.
 * tm_batch_status waits for `stream` and returns TM_OK or TM_EPRECISION for
 * everything launched since the last status read; rep->margin is the largest
 * rounding distance, rep->e_max the smallest bound of the batch's products.
 * tm_batch_destroy frees the batch (no launch of it may be in flight).
 * tm_mul_batch is the one-shot form: create, launch, wait, destroy.
 * Sources: Algorithms 1-3 per product; the batching has no counterpart in the
 * paper.
 */
typedef struct tm_desc {
  int32_t kind;           /* TM_FULL, TM_LO or TM_HI */
  int32_t reserved;       /* 0 */
  uint64_t n_bits;
  uint64_t* out;
  const uint64_t* u;
  const uint64_t* v;
} tm_desc;

typedef struct tm_batch tm_batch;

int tm_batch_create(tm_batch** batch, const tm_desc* descs, uint32_t count, void* stream);
int tm_batch_launch(tm_batch* batch, void* stream);
int tm_batch_status(tm_batch* batch, void* stream, tm_report* rep);
int tm_batch_destroy(tm_batch* batch);
int tm_mul_batch(const tm_desc* descs, uint32_t count, void* stream, tm_report* rep);

/*
 * Serving: a request queue with continuous batching under a device-memory
 * budget. Requests (kind, n_bits, DEVICE pointers as for tm_mul) are queued by
 * tm_server_submit and identified by the returned ticket (>= 0; a negative
 * value is a TM_E* code and nothing was queued). tm_server_progress never
 * blocks: it retires finished work (filling up to max_done completions with
 * their ticket and status), then admits queued requests, in arrival order,
 * into free slots: each slot is a CUDA stream, so admitted work overlaps on the
 * device with work already running. Consecutive small requests (transform
 * length N <= 4096) leave together as one launch of CTA-resident products;
 * a larger request takes a slot alone and is admitted only while the
 * workspaces of the requests in flight stay within budget_bytes (one request
 * is always admitted when nothing is in flight). Plan tables stay resident.
 * Results are bit-identical to tm_mul of the same request. Call from one
 * thread at a time per server (the calls lock). tm_server_pending returns the
 * number of requests queued or in flight; tm_server_destroy waits for the
 * work in flight and frees the server. The paper has no counterpart; this is
 * the library's serving layer.
 */
typedef struct tm_server tm_server;
typedef struct tm_completion {
  int64_t ticket;
  int32_t status;         /* TM_OK, TM_EPRECISION or TM_ECUDA */
  int32_t reserved;
} tm_completion;

int tm_server_create(tm_server** server, uint64_t budget_bytes, int slots);
int64_t tm_server_submit(tm_server* server, int kind, uint64_t* out, const uint64_t* u,
                         const uint64_t* v, uint64_t n_bits);
int tm_server_progress(tm_server* server, tm_completion* done, int max_done);
int tm_server_pending(tm_server* server);
int tm_server_destroy(tm_server* server);

/*
 * Kept operand transforms. The paper has no counterpart; it splits the
 * convolution of Algorithms 1-3 at its forward transforms. When one operand v is
 * multiplied by many u (a fixed Barrett reciprocal, a fixed modulus), its split,
 * forward map (alpha* for low, gamma-dagger with theta_V for high, none for full)
 * and forward FFT are computed once and kept on the device; each later product
 * then runs one forward map and one forward FFT, two transforms instead of three.
 *
 * tm_operand_create: plans (kind, n_bits), allocates the operand (8 N + 256
 * bytes of device memory, N the plan's transform length; tm_plan_query reports
 * N) and enqueues v's transform on `stream`. v is a device pointer with
 * ceil(n_bits/64) limbs; it is read by that enqueued work only and may be reused
 * once the stream has passed it. *out receives the handle (NULL on error). Use
 * the operand on the same stream, or order other streams after it (events).
 * tm_mul_operand: the product of the operand's kind and n_bits of u (device,
 * ceil(n_bits/64) limbs) and the kept v, into out (limb count as for tm_mul of
 * that kind). Same stream, status and rep conventions as tm_mul; TM_EINVAL when
 * the current device is not the one the operand was made on, TM_EALIAS when out
 * overlaps u. Results are bit-identical to tm_mul(kind, out, u, v, n_bits, ...).
 * tm_operand_destroy: frees the operand. No enqueued product may still read it.
 * The handle is not tied to the plan cache: tm_release() leaves it valid.
 * Returns TM_OK or a negative TM_E* code.
 */
typedef struct tm_operand tm_operand;
int tm_operand_create(int kind, uint64_t n_bits, const uint64_t* v, void* stream,
                      tm_operand** out);
int tm_mul_operand(uint64_t* out, const uint64_t* u, const tm_operand* v, void* stream,
                   tm_report* rep);
int tm_operand_destroy(tm_operand* op);

/*
 * Division by a k-bit divisor m (bit k-1 set, 1 <= k <= TM_MAX_BITS - 16), built on
 * the products above. The paper has no counterpart; its Section 1 names Barrett's
 * reduction as an application of the high product.
 *
 * tm_reciprocal: R = floor((2^(2k) - 1) / m) into R (device, ceil((k+1)/64)
 * limbs), m device with ceil(k/64) limbs. Newton's iteration for 1/m doubles the
 * precision h -> H <= 2h - 9 per step with one low product (E = 2^(H+h) - m_H X,
 * from its low H + 5 bits) and one high product (X E / 2^(2h)); the last step's
 * approximation is corrected exactly from e = 2^(2k) - 1 - m R (a low product mod
 * 2^(k+4)). Waits for the stream. Returns TM_OK, TM_EINVAL (NULL pointer, k = 0,
 * bit k-1 of m clear), TM_ERANGE, TM_ENOMEM, TM_ECUDA, or TM_EPRECISION (a product
 * on the stream failed its bound, or the final range check did not hold).
 *
 * tm_barrett_create: R = tm_reciprocal(m), plus kept transforms (tm_operand) of R
 * for high products of n = k + 1 bits and of m for low products of n = k + 3 bits,
 * plus scratch; about 40 k / 8 bytes of device memory. Waits for the stream. m
 * is read during the call only.
 * tm_barrett_divrem: q = floor(x / m) (ceil((k+1)/64) limbs) and r = x mod m
 * (ceil(k/64) limbs) for 0 <= x < 2^(2k) (ceil(2k/64) limbs; bits >= 2k ignored);
 * either output may be NULL, not both; outputs must not overlap x. Barrett's
 * quotient: x1 = floor(x / 2^(k-1)), q^ = the high product of x1 and R (n = k + 1),
 * so q - 3 <= q^ <= q + 1; r^ = x - q^ m from x and the low product of q^ and m
 * (n = k + 3), then at most one addition and three subtractions of m, taken on
 * the device by sign tests. Enqueued on `stream`; rep as for tm_mul: the high
 * product's plan, e_max the larger bound of the two products and margin the
 * largest rounding distance of both (with rep, TM_EPRECISION also reports a
 * failed final range check 0 <= r < m). Calls on one
 * context share its scratch: order them on one stream.
 * tm_barrett_reciprocal: copies R (ceil((k+1)/64) limbs, device) on `stream`.
 * tm_barrett_destroy: waits for the device, then frees the context.
 */
typedef struct tm_barrett tm_barrett;
int tm_reciprocal(uint64_t* R, const uint64_t* m, uint64_t k_bits, void* stream);
int tm_barrett_create(const uint64_t* m, uint64_t k_bits, void* stream, tm_barrett** out);
int tm_barrett_divrem(tm_barrett* b, uint64_t* q, uint64_t* r, const uint64_t* x, void* stream,
                      tm_report* rep);
int tm_barrett_reciprocal(const tm_barrett* b, uint64_t* R, void* stream);
int tm_barrett_destroy(tm_barrett* b);

/*
 * tm_coeffs: the rounded coefficients c_i of one product (device pointers),
 * for checking the method stage by stage:
 *   low:  c_i = round(2^b Wbar_i) = 2^b L_i, i < N       (Algorithm 2,
 *         Proposition 3.1);
 *   high: c_i = round(2^b Wbar_i) = 2^b H_i, i <= N      (Algorithm 3,
 *         Proposition 4.1);
 *   full: c_i = round(Wbar_i) = w_i, i < N (the cyclic length) (Algorithm 1).
 * c_out must hold rep->n_digits (high: N + 1) or N int64 values: use
 * tm_plan_query first. Waits for the stream; *rep is required.
 */
int tm_coeffs(int kind, int64_t* c_out, const uint64_t* u, const uint64_t* v, uint64_t n_bits,
              void* stream, tm_report* rep);

/*
 * tm_autotune: picks the FFT pass layout for the transform length of (kind,
 * n_bits) by measurement. Candidates vary the points per CTA, how the odd prime
 * factors of the length are spread over the passes, and the number of passes; each
 * is timed on `stream` (two forward transforms and one inverse, CUDA events, median
 * of five after a warm-up, each behind a short device-side delay so that the host's
 * launches are not timed) on scratch buffers of 4 x 16 (N/2) bytes allocated for
 * the call. The fastest, if at least 1% faster than the default layout (else the
 * default), becomes the layout of every later plan with that length on
 * this device (plans built before keep theirs for their current users, e.g. a
 * tm_batch). Results of products do not depend on the layout (they are exact);
 * only the time does. Waits for the stream. *out: candidates timed, the chosen
 * layout, its pass count, and the default and chosen layouts' times (ms).
 */
typedef struct tm_tune {
  int32_t candidates;
  int32_t points;      /* points per CTA the chosen layout aims for        */
  int32_t split;       /* 0 balanced, 1 odd primes first pass, 2 last pass */
  int32_t passes;      /* 0 default count, else 2 or 3                     */
  int32_t npass;       /* passes of the chosen layout                      */
  int32_t reserved;
  double ms_default;
  double ms_best;
} tm_tune;
int tm_autotune(int kind, uint64_t n_bits, void* stream, tm_tune* out);

/*
 * tm_set_layout: makes a layout (points, split and passes of *layout, as
 * tm_autotune reports them; the other fields are ignored) the FFT pass layout of
 * every later plan with the transform length of (kind, n_bits) on the current
 * device, without timing anything: a layout chosen by tm_autotune in an earlier
 * process can be reapplied. points, split and passes as in tm_tune (points
 * 32..4096); points 1024, split 0, passes 0 is the default layout.
 * Results do not depend on the layout. Errors: TM_EINVAL (bad kind, n_bits = 0,
 * null layout or a field out of range), TM_ERANGE (n_bits too large, or no valid
 * pass split of the length with that many passes), TM_ECUDA (no device).
 */
int tm_set_layout(int kind, uint64_t n_bits, const tm_tune* layout);

/*
 * tm_autotune_plan: picks the plan (b, N) of (kind, n_bits) by measurement, as
 * the paper's Section 5 picks N among its candidate lengths by their timings.
 * Candidates: every certified plan (worst-case bound within the target, so every
 * result stays exact) whose transform length is at most 1.15x the planner's, the
 * planner's first, at most 8. Each candidate runs with the FFT layout set for its
 * transform length (the default unless tm_autotune or tm_set_layout set one); it runs
 * whole products on scratch operands on `stream` (one warm-up, then the median of
 * five CUDA-event timings of one product each, behind a short device-side delay so
 * that the host's planning and launch work is not timed); the fastest, if at least 1%
 * faster than the planner's (else the planner's), becomes the plan of (kind, n_bits)
 * for later calls in this process (tm_mul and the calls
 * built on it; tm_mul_static keeps the planner's). Low and full products do not
 * change; a high product may become the other admissible value. Tables of the
 * losing candidates are freed. Waits for the stream. *out: the chosen b and N,
 * the number of candidates, and the planner's and the chosen plan's times (ms).
 * Errors: TM_EINVAL, TM_ERANGE as tm_mul; TM_ENOMEM for the scratch operands.
 */
typedef struct tm_plan_tune {
  uint32_t b;
  uint32_t N;
  uint32_t candidates;
  uint32_t reserved;
  double ms_default;
  double ms_best;
} tm_plan_tune;
int tm_autotune_plan(int kind, uint64_t n_bits, void* stream, tm_plan_tune* out);

/*
 * tm_plan_set: makes the certified plan (b, N) the plan of (kind, n_bits) for later
 * calls in this process (for example one chosen by tm_autotune_plan earlier; as
 * there, tm_mul_static keeps the planner's); b = N = 0 restores the planner's choice. TM_EINVAL for parameters outside the
 * ranges of tm_mul_params, TM_ERANGE when the worst-case bound for (b, N) is above
 * the target (use tm_mul_params for uncertified parameters).
 */
int tm_plan_set(int kind, uint64_t n_bits, uint32_t b, uint32_t N);

/*
 * tm_plan_query: the plan the library uses for (kind, n_bits), without any
 * device work: fills b, N, n_digits, lam_fwd, lam_bwd, fft_passes, fwd_streams,
 * e_max and workspace_bytes of *rep (fwd_streams from the current device's SM
 * count, 152 without a device). Host only. Returns TM_OK, TM_EINVAL or TM_ERANGE.
 */
int tm_plan_query(int kind, uint64_t n_bits, tm_report* rep);

/*
 * tm_stream_status: waits for `stream`, then returns and clears the
 * device-side status accumulated by asynchronous calls on it (TM_OK or
 * TM_EPRECISION); if rep != NULL, rep->margin receives the largest margin
 * seen since the last clear.
 */
int tm_stream_status(void* stream, tm_report* rep);

/* tm_release: frees every plan table and workspace of the current device.
 * No call may be in flight on that device. */
int tm_release(void);

/*
 * tm_set_fused: how products run. A product is either a sequence of per-phase
 * kernel launches (maps, FFT passes, twist, back map, carry scan), or one
 * cooperative launch that runs the same phases with grid-wide barriers between
 * them, which removes the launch gaps that dominate small and medium sizes. The
 * arithmetic is the same, so the results are identical.
 *   mode 0  automatic (the default): per-phase launches, and batches as a
 *           graph of per-phase launches (measured faster on GB300: a grid
 *           barrier costs about as much as a launch gap, and the 4096-product
 *           batch takes 29 ms as one persistent launch against 19.5 ms);
 *   mode 1  always per-phase launches (the same as mode 0 in this version);
 *   mode 2  one cooperative launch per single product, and every batch created
 *           afterwards as one persistent launch under a one-node CUDA graph,
 *           whenever the FFT layout allows it (sub-transforms of at most 2048
 *           points).
 * Applies to tm_mul and the calls built on it and to batches created afterwards
 * (process wide). tm_mul_events, tm_coeffs and kept operands always use
 * per-phase launches.
 * The barrier waits are bounded: a wait that gives up (about a second) makes the
 * call report TM_ETIMEOUT instead of hanging. No counterpart in the paper.
 * Returns TM_OK or TM_EINVAL.
 */
int tm_set_fused(int mode);

/*
 * tm_convolution: the Convolution step of Section 2.1 on its own - the cyclic
 * convolution out = x * y of two real sequences of length N in FP64, computed by
 * the same kernels as the products (two forward FFTs of the packed sequences, the
 * fused twist and pointwise product, one inverse FFT).
 *   out, x, y  device arrays of N doubles; out must not overlap x or y (x == y is
 *              allowed).
 *   N          a transform length the products use: even, 2^a m with m one of the
 *              odd parts listed for tm_mul_params, 4 <= N <= 2^31.
 *   eta        optional (NULL): receives the error bound of this computation:
 *              |out_k - (x*y)_k| <= eta ||x||_2 ||y||_2 for every k, derived for
 *              the kernels' arithmetic (every FFT pass layout).
 * Asynchronous on `stream`; uses the stream's workspace and the length's tables.
 * Returns TM_OK, TM_EINVAL, TM_ENOMEM or TM_ECUDA.
 */
int tm_convolution(double* out, const double* x, const double* y, int64_t N, void* stream,
                   double* eta);

/*
 * tm_table_values: writes the twiddle tables the FFT kernels use into the
 * caller's device buffer `out` (enqueued on `stream`), so that their accuracy can
 * be checked; a checking facility with no counterpart in the paper.
 *   which 0: out[2m], out[2m+1] = cos, -sin of 2 pi m / len, m < count;
 *   which 1: the tangent-form records of a radix-4 stage with Ns = len
 *            (count must equal len): out[4k..4k+3] = t1, c1, t2, c2s with
 *            exp(-2 pi i k / (4 len)) = c1 (1 - i t1) and exp(-4 pi i k / (4 len))
 *            = c2 (1 - i t2), or -i c2 (1 - i t2) with c2s = -c2 when its angle
 *            is pi/2 or more;
 *   which 2: the twist coefficients of real length N = len: out[2k], out[2k+1]
 *            = cos(2 pi k / N) (cos, -sin)(2 pi k / N) / N, k < count;
 *   which 3: the four-step twiddles of a pass with Mp = len and Qc = count
 *            sequences (count must divide len), in the pass's output order:
 *            out[2e], out[2e+1] = cos, -sin of 2 pi (qc k mod Mp) / Mp at
 *            e = k Qc + qc, qc < Qc, k < len / count (len entries).
 * Each value is the double nearest to the exact one, up to 2^-40 of an ulp
 * (the tangent t is nearest to sin / c with the stored c). Returns TM_OK,
 * TM_EINVAL or TM_ECUDA.
 */
int tm_table_values(int which, int64_t len, int64_t count, double* out, void* stream);

/*
 * tm_probe_dfma: a measurement helper with no counterpart in the paper. Enqueues
 * on `stream` one kernel that keeps every SM's FP64 pipe busy with independent
 * fused multiply-adds (8 CTAs of 256 threads per SM, 8 chains of `iters` FMAs per
 * thread) and stores the flops it performs (2 per FMA) in *flops; the caller
 * times it with events on the stream. The FP64 pipe bounds the FFT passes, so
 * flops / time is the peak their roofline fraction is taken against. Returns
 * TM_OK, TM_EINVAL (iters <= 0, NULL flops) or TM_ECUDA.
 */
int tm_probe_dfma(int iters, void* stream, double* flops);

/* Text for a status code (static storage). */
const char* tm_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* TRUNCMUL_H */

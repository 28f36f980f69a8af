/*
 * neumann.h - C ABI of the GB300 (sm_103a) truncated Neumann series library.
 *
 * Computes S_k(A) = I + A + A^2 + ... + A^{k-1} for a dense n x n matrix A
 * with spectral radius rho(A) < 1 (Sec. 1, Eq. neumann; Sec. 2, Eq. series),
 * by one of the paper's schemes:
 *   radix 1   naive accumulation of powers, k-2 products      (Sec. 2.1)
 *   radix 2   repeated squaring (k = 2^t), or the binary digits of k with
 *             NEUMANN_FLAG_EXACT_K                             (Sec. 2.1)
 *   radix 3,5 exact ternary / quinary kernels                  (Sec. 2.1, Sec. 2.3)
 *   radix 9   exact 3-product radix-9 kernel, k = 9^t          (Thm 3.1)
 *   radix 15  approximate 4-product radix-15 kernel inside the residual
 *             framework, k = 15^t                             (Sec. 4, Sec. 5.3)
 *   radix 24, 25, 27, 31, 33  approximate 5-product kernels inside the residual
 *             framework, k = m^t: the Sec. 4.1 circuit with a fifth product, at
 *             the 5-product budget of App. C (Table approx). The circuits are the
 *             library's own: exact prefix [T~]_j = 1 for j < m at 24 and 25,
 *             least-squares prefixes at 27, 31, 33 (neumann_radix_p5_coefficients).
 *             Radix 33 converges for real eigenvalues in (-0.925, 1) only
 *   radix 0   exact kernels over the factorisation of k into 9, 5, 3, 2
 *             (block concatenation, Sec. 2.2, eq. decomposition); with
 *             NEUMANN_FLAG_ALLOW_APPROX also radix-15 levels (Lemma 5.7 holds
 *             level by level, Sec. 5.3)
 * Every level applies a kernel f to the current residual R (R_0 = A), updates
 * the partial sum Y <- Y f(R) (Y_0 = I) and the residual R <- I - (I - R) f(R)
 * (Sec. 5.3, eq. generalradix and the proof of Lemma 5.7). For an exact
 * kernel f = T_m this residual is the next power A^{m n} (telescoping,
 * Sec. 2.2), so all schemes share one level loop.
 *
 * Result of radix 15, 24, 25, 27, 31 and 33: the residual-framework value
 * Y_t = (I-A)^{-1}(I - E^[t](A)) of Lemma 5.7, which agrees with S_k through the
 * degree-(k-1) term.
 *
 * Arithmetic (neumann_dtype_t):
 *   FP64        every product in FP64 on the CUDA cores; A and S are double.
 *   FP32        every product in FP32 on the CUDA cores; the partial sum Y and
 *               the residual R are accumulated in FP64; A and S are float.
 *   SPLIT_BF16  every product on the tcgen05 tensor cores from hi+lo BF16
 *               operands (x = hi + lo, three products hi*hi + hi*lo + lo*hi,
 *               FP32 accumulation in tensor memory); Y and R accumulated in
 *               FP64. A and S are double unless NEUMANN_FLAG_IO_FP32.
 *   SPLIT_FP16  as SPLIT_BF16 with FP16 hi+lo operands of x * 2^e, e chosen per
 *               matrix (and per matrix of a batch) so that a bound on its max |x|
 *               maps to 2^14: x = hi + lo to ~2^-22 relative for entries within
 *               ~2^-17 of that bound, ~2^-39 of the bound absolute below. The
 *               bound comes from max |x| and column sums measured by the
 *               producing launches; FP16 overflow cannot occur unless an input
 *               is not finite.
 *
 * Conventions shared by every call:
 *   - Matrices are dense, row-major, n x n, with a leading dimension (in
 *     elements, >= n) given per pointer. Device pointers are CUDA device
 *     memory of the current device; host pointers are named as such.
 *   - `stream` is a cudaStream_t passed as void*; NULL is the legacy default stream.
 *   - Calls return NEUMANN_OK (0) or an error code below; nothing throws.
 *   - Work is stream-ordered and asynchronous: a call returns once its kernels
 *     are queued. Conditions detected on the device (non-finite values,
 *     a bounded wait that expired) are read with neumann_last_status.
 *   - Precondition rho(A) < 1 is documented, not checked. Radix 15 converges
 *     for real eigenvalues |l| < ~0.97.
 */
#ifndef NEUMANN_GB300_H
#define NEUMANN_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct neumann_plan_s* neumann_plan_t;

typedef enum {
  NEUMANN_FP64 = 0,
  NEUMANN_FP32 = 1,
  NEUMANN_SPLIT_BF16 = 2,
  NEUMANN_SPLIT_FP16 = 3
} neumann_dtype_t;

/* Return codes. */
#define NEUMANN_OK 0
#define NEUMANN_EINVAL 1  /* bad argument: n < 1, k < 1, k not a power of the radix, ld < n, aliasing, NULL */
#define NEUMANN_ENOMEM 2  /* device or host allocation failed */
#define NEUMANN_ECUDA 3   /* a CUDA call or kernel launch failed */
#define NEUMANN_ENOTSUP 4 /* dtype / radix combination not supported */

/* Device status bits reported by neumann_last_status. */
#define NEUMANN_STATUS_NONFINITE 1u /* an epilogue produced Inf/NaN (in practice rho(A) >= 1) */
#define NEUMANN_STATUS_TIMEOUT 2u   /* a bounded device wait expired; the result is invalid */

/* Plan flags. */
#define NEUMANN_FLAG_EXACT_K 0x1u         /* radix 2: any k >= 1 by the binary digits of k */
#define NEUMANN_FLAG_RESIDUAL_PAPER 0x2u  /* residual R' = I - (I - A) Y' (eq. generalradix) instead of R' = R + R G - G */
#define NEUMANN_FLAG_PRINTED_COEFFS 0x4u  /* radix 15: the three-decimal coefficients printed in App. B */
#define NEUMANN_FLAG_TIMING 0x8u          /* record CUDA events around every product (neumann_plan_timing) */
#define NEUMANN_FLAG_IO_FP32 0x10u        /* split dtypes: A and S are float instead of double */
#define NEUMANN_FLAG_SINGLE_CTA 0x20u     /* split dtypes: keep every product on single-CTA 128 x 256 tiles
                                             (by default padded orders >= 4096 use 2-CTA 256 x 256 tiles) */
#define NEUMANN_FLAG_SYMMETRIC 0x80u      /* single plans: A is symmetric, so is every matrix of the scheme (each
                                             is a polynomial in A): products compute only the tiles on or above
                                             the diagonal (256 x 256 CTA pairs for split dtypes, 128 x 128 for
                                             FP64/FP32) and write their transposes; split right operands are
                                             read from the row-major hi/lo pairs. About half the product work.
                                             A must be symmetric (the result is otherwise unspecified); S is
                                             exactly symmetric. Not with NEUMANN_FLAG_PRECISE_ACC; ignored by
                                             grouped batches */
#define NEUMANN_FLAG_PRECISE_ACC 0x40u    /* split dtypes: products accumulate K in chunks of 512, each chunk
                                             added to the running FP32 sum with round-to-nearest. The tensor
                                             cores' accumulator rounds every update toward zero, a bias of about
                                             (3K/16)/4 ulp over a K-long sum; chunking bounds the truncated chain
                                             to 96 updates. 2-CTA 256 x 128 tiles; slower. Single plans only
                                             (a grouped batch's K is at most 256) */

#define NEUMANN_FLAG_ALLOW_APPROX 0x100u /* radix 0: k = 2^a 3^b 5^c is split into the levels of least product
                                             count over the exact kernels 2, 3, 5, 9 AND the approximate radix-15
                                             kernel (ties: fewer radix-15 levels, then fewer levels); exact levels
                                             run first, radix-15 levels last. The result is then the residual-
                                             framework value of Lemma 5.7 for that level sequence, which agrees
                                             with S_k through degree k-1 */

#define NEUMANN_FLAG_NO_RESIDENT 0x200u  /* batched plans: run every matrix through the grouped launches (by
                                             default the batch's matrices of order <= info.resident_max_n run in
                                             one launch that keeps each matrix's whole level loop in one CTA's
                                             shared memory) */

#define NEUMANN_MAX_LEVELS 64

typedef struct {
  int64_t n, k;
  int radix;                    /* as requested */
  int dtype;                    /* neumann_dtype_t */
  uint32_t flags;
  int levels;                   /* radix levels (0 for the naive chain and for k <= 2) */
  int level_radix[NEUMANN_MAX_LEVELS];
  int64_t products_formula;     /* the paper's count: k-1 (naive), 2 ceil(log2 k) (binary, Sec. 6),
                                   sum of mu_m + 2 over levels (Sec. 2.2 cost model) */
  int64_t products_executed;    /* products this plan launches (no product with I, no unused power) */
  int64_t launches;             /* kernel launches per neumann_eval */
  size_t workspace_bytes;       /* device workspace the plan needs */
  int64_t padded_n;             /* workspace matrices are padded_n x padded_n */
  /* Launch configuration (set by neumann_plan_autotune*, else the defaults): */
  int tile_pair;                /* split dtypes, single plans: 1 = products on 2-CTA 256 x 256 tiles,
                                   0 = 1-CTA 128 x 256 tiles */
  int raster_group;             /* split dtypes, single plans: row tiles per raster group */
  int batch_chunk;              /* grouped batched plans (max_n <= 256): matrices per pass */
  int tuned;                    /* 1 once tuned, by this plan or by an earlier plan of the same shape */
  /* Algorithmic device-memory bytes per matrix element (x n^2 for one evaluation,
     x sum n_i^2 for a batch): every input and output representation of every
     launch read or written once, plus both operands of each product. */
  int64_t bytes_per_element;          /* all launches of an evaluation */
  int64_t product_bytes_per_element;  /* the products alone */
  int resident_max_n;           /* grouped batched plans: matrices of order <= this run in the resident
                                   launch: 48 untuned (at most what one CTA's shared memory holds, 52-60
                                   by scheme), then as neumann_plan_autotune_batched picks it (0: none,
                                   FP64 plans, or NEUMANN_FLAG_NO_RESIDENT) */
} neumann_plan_info_t;

/* Create a plan for S_k(A) with A n x n. Host-only: no device memory is
 * touched. The plan owns a device workspace of info.workspace_bytes that is
 * allocated on the first neumann_eval unless the caller supplies one with
 * neumann_plan_set_workspace.
 *   out    receives the plan (set to NULL on error)
 *   n      matrix order, >= 1
 *   k      number of series terms, >= 1; for radix 3, 5, 9, 15, 24, 25, 27, 31, 33 a power of the radix;
 *          for radix 2 a power of two unless NEUMANN_FLAG_EXACT_K; for radix 0 of the
 *          form 2^a 3^b 5^c (levels as NEUMANN_FLAG_ALLOW_APPROX says)
 *   radix  0, 1, 2, 3, 5, 9, 15, 24, 25, 27, 31 or 33 (see above)
 *   dtype  neumann_dtype_t
 *   flags  NEUMANN_FLAG_*
 * Errors: NEUMANN_EINVAL, NEUMANN_ENOTSUP, NEUMANN_ENOMEM (host). */
int neumann_plan_create(neumann_plan_t* out, int64_t n, int64_t k, int radix, int dtype, uint32_t flags);

/* Fill *info for a plan. Errors: NEUMANN_EINVAL (NULL). */
int neumann_plan_info(neumann_plan_t plan, neumann_plan_info_t* info);

/* Give the plan a caller-owned device workspace of at least
 * info.workspace_bytes bytes, 256-byte aligned. The caller keeps ownership and
 * must keep it alive until the plan is destroyed or another workspace is set.
 * No initial contents are required: the call clears the device status word (the
 * first 256 bytes, synchronously) and every evaluation rewrites each buffer it
 * reads, padding included. Errors: NEUMANN_EINVAL (too small, misaligned),
 * NEUMANN_ECUDA. */
int neumann_plan_set_workspace(neumann_plan_t plan, void* workspace, size_t bytes);

/* S <- S_k(A) for the plan's n, k, radix and dtype.
 *   A    device, n x n row-major, leading dimension lda >= n (double for FP64 and
 *        split dtypes, float for FP32 and with NEUMANN_FLAG_IO_FP32); read only
 *   S    device, n x n row-major, leading dimension lds >= n, same element type as A;
 *        must not overlap A
 * Stream-ordered. Allocates the workspace with cudaMalloc on first use when none
 * was set. Two evaluations with the same plan must not run concurrently.
 * Errors: NEUMANN_EINVAL, NEUMANN_ENOMEM, NEUMANN_ECUDA. */
int neumann_eval(neumann_plan_t plan, const void* A, int64_t lda, void* S, int64_t lds, void* stream);

/* S <- S_k(A) for matrices in HOST memory: the call copies A into one of two
 * plan-owned device staging sets on the plan's input copy stream, evaluates on
 * `stream`, and copies the result to S on the plan's output copy stream. It
 * returns once that work is enqueued. Consecutive calls alternate between the
 * two sets, so one call's copy-in and the previous call's copy-out run while an
 * evaluation runs.
 *   A, S  host, n x n row-major with leading dimensions lda, lds >= n, element type
 *         as in neumann_eval. Pinned memory (cudaHostAlloc / cudaHostRegister) gives
 *         asynchronous copies; pageable memory is copied synchronously by the driver.
 *         A must stay unchanged and S unread until neumann_plan_host_wait returns.
 * The first call allocates the staging sets (4 n^2 elements) and the streams.
 * Errors: NEUMANN_EINVAL (batched plan, bad arguments, A and S overlap),
 * NEUMANN_ENOMEM, NEUMANN_ECUDA. */
int neumann_eval_host(neumann_plan_t plan, const void* A, int64_t lda, void* S, int64_t lds, void* stream);

/* S_i <- S_k(A_i), i < count, for a batch PACKED in host memory: matrix i
 * (n_i x n_i, row-major, leading dimension n_i) starts at element
 * sum_{j<i} n_j^2 of A and of S. The call copies the packed batch into one
 * plan-owned device staging pair on the plan's input copy stream, evaluates it
 * on `stream` (as neumann_eval_batched), and copies the results out on the
 * plan's output copy stream; it returns once that work is enqueued. The next
 * call's copy-in waits only for the last step that reads A, and its first write
 * of S only for this call's copy-out, so copies overlap evaluations.
 * Host buffers as in neumann_eval_host (pinned for asynchronous copies; stable
 * until neumann_plan_host_wait). The staging pair grows to the largest batch
 * seen (2 x sum n_i^2 elements). Errors as neumann_eval_batched. */
int neumann_eval_batched_host(neumann_plan_t plan, int count, const int64_t* n, const void* A, void* S,
                              void* stream);

/* Block until every copy issued by neumann_eval_host / neumann_eval_batched_host on this plan has completed
 * (results in host memory, inputs no longer read). Errors: NEUMANN_EINVAL,
 * NEUMANN_ECUDA. */
int neumann_plan_host_wait(neumann_plan_t plan);

/* C <- A B in the plan's arithmetic (the product every scheme step uses), for
 * n x n row-major device matrices with leading dimension n, element type as in
 * neumann_eval. Uses the plan's workspace for split operands. Stream-ordered.
 * Errors as neumann_eval. */
int neumann_plan_matmul(neumann_plan_t plan, const void* A, const void* B, void* C, void* stream);

/* Batched plan: `count` independent evaluations with n_i <= max_n, the same k,
 * radix and dtype. Host-only, like neumann_plan_create. */
int neumann_plan_create_batched(neumann_plan_t* out, int count, int64_t max_n, int64_t k, int radix,
                                int dtype, uint32_t flags);

/* S_i <- S_k(A_i), i < count.
 * Matrices of order <= info.resident_max_n (at most 64) run in one persistent
 * launch, largest first, each through the whole scheme inside one CTA's shared
 * memory (FP64 partial sums in a per-CTA scratch); the others in grouped
 * launches, one per op of the scheme over up to 2048 matrices at a time.
 *   n  HOST array of count orders (1 <= n_i <= max_n)
 *   A  HOST array of count device pointers (n_i x n_i, leading dimension n_i)
 *   S  HOST array of count device pointers (same shapes; no overlap with any A_j)
 * Stream-ordered. Errors: NEUMANN_EINVAL (count or n_i out of range),
 * NEUMANN_ENOMEM, NEUMANN_ECUDA. */
int neumann_eval_batched(neumann_plan_t plan, int count, const int64_t* n, const void* const* A,
                         void* const* S, void* stream);

/* Synchronise the plan's last stream and return the OR of the device status
 * bits (NEUMANN_STATUS_*) set since the previous call, then clear them.
 * Errors: NEUMANN_EINVAL, NEUMANN_ECUDA. */
int neumann_last_status(neumann_plan_t plan, unsigned* status);

/* Autotuner. Times each candidate launch configuration on the caller's input
 * (one untimed and `reps` timed evaluations per candidate, CUDA events on the
 * stream, median), keeps the fastest in the plan and records it for the
 * process: plans created later with the same shape start from it (their
 * info.tuned is 1). The evaluations write S (its final contents are those of a
 * correct evaluation). Synchronous: returns after the last timed run.
 *   split dtypes   candidates: {1-CTA, 2-CTA pair} tiles x raster groups {4, 8, 16}
 *                  (pairs are skipped under NEUMANN_FLAG_SINGLE_CTA); shape key
 *                  (padded_n, dtype)
 *   FP64, FP32     one launch shape: marks the plan tuned and returns
 * Arguments as neumann_eval; reps >= 1.
 * Errors: NEUMANN_EINVAL (batched plan, bad arguments), NEUMANN_ENOMEM, NEUMANN_ECUDA. */
int neumann_plan_autotune(neumann_plan_t plan, const void* A, int64_t lda, void* S, int64_t lds, int reps,
                          void* stream);

/* Set a split-dtype single plan's launch configuration by hand, as
 * neumann_plan_autotune would: tile_pair -1 (CTA pairs from padded order 4096),
 * 0 (1-CTA tiles) or 1 (2-CTA pairs; ignored under NEUMANN_FLAG_SINGLE_CTA,
 * and precise or symmetric plans always use pairs); raster_group 1 .. 65535
 * row tiles. Marks the plan tuned without recording the choice for other
 * plans. Host-only (re-encodes the tensor maps of an attached workspace; no
 * launch, no synchronisation).
 * Errors: NEUMANN_EINVAL (batched, FP32 or FP64 plans; values out of range),
 * NEUMANN_ECUDA (tensor-map encoding). */
int neumann_plan_set_launch(neumann_plan_t plan, int tile_pair, int raster_group);

/* Autotuner for a batched plan: arguments as neumann_eval_batched plus reps.
 * For a grouped plan (max_n <= 256) it times first the largest order the
 * resident launch takes (0, 16, 32, 48 and the most it holds; the rest run
 * grouped), then the number of matrices per grouped pass (the plan's chunk
 * halved down to 64, at most 6 candidates): smaller passes keep a pass's
 * intermediate matrices in L2, larger ones fill the GPU with fewer launches. Shape key (count, max_n, k, radix, dtype). A plan with larger
 * orders runs one single plan per order and is only marked tuned.
 * Errors as neumann_eval_batched. */
int neumann_plan_autotune_batched(neumann_plan_t plan, int count, const int64_t* n, const void* const* A,
                                  void* const* S, int reps, void* stream);

/* With NEUMANN_FLAG_TIMING every product launched by neumann_eval is bracketed
 * by two CUDA events on the evaluation's stream (not while the stream is being
 * captured into a CUDA graph: a captured evaluation records nothing). This call synchronises on the
 * last of them, copies the device time (ms) of each product recorded since the
 * previous call into ms[0..cap-1] (in launch order), sets *count to the number
 * recorded, and starts a new record. At most 65536 products are kept; an
 * evaluation that would exceed that returns NEUMANN_EINVAL.
 * Errors: NEUMANN_EINVAL (no timing flag), NEUMANN_ECUDA. */
int neumann_plan_timing(neumann_plan_t plan, float* ms, int cap, int* count);

/* Self-test of device failure reporting: launches one thread that waits, with
 * the same bounded-wait code the tensor-core product uses, on an mbarrier that
 * nothing arrives on, for limit_ns nanoseconds (at most 1e9), and then sets
 * NEUMANN_STATUS_TIMEOUT in the plan's status word (read with neumann_last_status).
 * No kernel faults or hangs: the wait ends by itself and the context stays usable.
 * Stream-ordered. Errors: NEUMANN_EINVAL, NEUMANN_ENOMEM, NEUMANN_ECUDA. */
int neumann_plan_selftest_timeout(neumann_plan_t plan, uint64_t limit_ns, void* stream);

/* The 28 radix-15 circuit parameters the library uses (Sec. 4.1, App. B), in
 * the order l2[3], r2[3], l3[4], r3[4], l4[5], r4[5], gamma[4]; set 0 = refined
 * on the host by minimum-norm Gauss-Newton from the printed values, 1 = as printed.
 * Also returns max_{j<15} |[T~15]_j - 1| and the spillover [T~15]_15, [T~15]_16.
 * Errors: NEUMANN_EINVAL. */
int neumann_radix15_coefficients(int set, double* coef28, double* prefix_error, double* spill15,
                                 double* spill16);

/* The 41 parameters of the five-product kernel of radix m = 24, 25, 27, 31 or 33
 * that the library uses. Circuit: P1 = B^2; for i = 2..5, L_i and R_i are linear
 * combinations over (I, B, P1, ..., P_{i-1}) and P_i = L_i R_i;
 * T~ = I + g1 B + g2 P1 + g3 P2 + g4 P3 + g5 P4 + P5 (Sec. 4.1 structure, one more
 * product; App. C, Table approx). Order: l2[3], r2[3], l3[4], r3[4], l4[5], r4[5],
 * l5[6], r5[6], gamma[5]. The values are the minimum-norm Gauss-Newton solution
 * of the m prefix equations [T~]_j = 1, j < m, from the library's published
 * six-decimal circuit, refined on the host on first use (m = 24, 25: exact
 * prefix); for m = 27, 31, 33 no exact prefix exists in the library's search and
 * the kernel is a published least-squares point used as it is (kernel residual
 * sum_{j<m} ([T~]_j - 1)^2 = 4.7e-4, 0.109, 0.554; App. C, Table approx).
 *   coef41        receives the parameters (caller-owned, 41 doubles)
 *   prefix_error  receives max_{j<m} |[T~]_j - 1| (may be NULL)
 *   spill         receives the spillover [T~]_m (may be NULL)
 * Errors: NEUMANN_EINVAL (m not 24, 25, 27, 31 or 33; coef41 NULL), NEUMANN_ENOTSUP
 * (the refinement of 24 / 25 did not reach rounding level). */
int neumann_radix_p5_coefficients(int m, double* coef41, double* prefix_error, double* spill);

/* C <- A B without any device allocation. The paper has no counterpart to this
 * call; it exists for callers that cannot call cudaMalloc/cudaFree where they
 * need a product: code running under an allocator that owns all device memory
 * (a framework's caching allocator, an allocation hook that must not re-enter
 * the driver's allocator) and latency-critical loops that cannot take the
 * device-wide synchronisation cudaFree implies. Such callers cannot give a plan
 * a workspace, nor let neumann_plan_matmul allocate one.
 * Arithmetic and kernels are those of neumann_plan_matmul on a
 * NEUMANN_SPLIT_BF16 plan (hi/lo BF16 operands, three tensor-core products,
 * FP32 accumulation); the scratch (a status word and the hi/lo operands) is a
 * fixed device array of 8 MiB + 256 bytes inside the library, present on every
 * GPU that loads the library's code until the process exits.
 *   n      order, 1 <= n <= 1024; larger n returns NEUMANN_EINVAL
 *   A, B   device, double, n x n row-major, leading dimensions lda, ldb >= n; read only
 *   C      device, double, n x n row-major, leading dimension ldc >= n; must not
 *          overlap A or B
 *   stream a stream of the current device
 * Stream-ordered. Set-up: under CUDA's default lazy module loading, the first
 * call on a device loads the library's device code into that device's context,
 * which is when the driver reserves the 8 MiB array (and the kernels' own
 * memory); that load may synchronise the device. Make the first call in set-up
 * code, before any stream capture and outside any allocator hook; later calls
 * only look up the array's address (a runtime table query, no allocation).
 * Every call on a device shares the array: calls whose work overlaps on the
 * GPU (different streams, different host threads) race and must be serialised
 * by the caller. Device status bits (a non-finite result, an expired bounded
 * wait) are OR-ed into the array's status word; read them with
 * neumann_matmul_noalloc_status.
 * Errors: NEUMANN_EINVAL, NEUMANN_ECUDA. */
int neumann_matmul_noalloc(int64_t n, const void* A, int64_t lda, const void* B, int64_t ldb, void* C,
                           int64_t ldc, void* stream);

/* Synchronise `stream` (of the current device), return in *status the OR of
 * the NEUMANN_STATUS_* bits that neumann_matmul_noalloc calls on this device
 * set since the previous read, and clear them. Allocates nothing. The paper
 * has no counterpart to this call.
 * Errors: NEUMANN_EINVAL (status NULL), NEUMANN_ECUDA. */
int neumann_matmul_noalloc_status(void* stream, unsigned* status);

/* Measurement aid (no counterpart in the paper): the CUDA cores' FMA rate of
 * the current device in TFLOP/s, for dtype NEUMANN_FP32 or NEUMANN_FP64, from
 * timed launches (CUDA events on `stream`, best of three after a warm-up) of a
 * kernel whose threads run 8 independent FMA chains, 2048 threads per SM. It is
 * the roofline denominator of the FP32 and FP64 product kernels. *sms (may be
 * NULL) receives the device's SM count. Synchronises `stream`; allocates nothing.
 * Errors: NEUMANN_EINVAL, NEUMANN_ECUDA. */
int neumann_measure_fma_peak(int dtype, double* tflops, int* sms, void* stream);

/* Release a plan and the workspace it allocated (not a caller-set one). NULL is ignored. */
void neumann_plan_destroy(neumann_plan_t plan);

/* Static string for a return code. */
const char* neumann_error_string(int code);

#ifdef __cplusplus
}
#endif

#endif /* NEUMANN_GB300_H */

/*
 * liblpdec -- ADMM LP decoding of LDPC codes on a GB300 (sm_103a) GPU.
 *
 * The method is Algorithm 1 of "Decomposition Methods for Large Scale LP
 * Decoding" (Barman, Liu, Draper, Recht), Section 3.3: the alternating
 * direction method of multipliers applied to Feldman's LP relaxation
 * (Section 2, eq. (feldmanLP)), with the check-side z-update computed by the
 * two-slice projection onto the parity polytope (Section 4.4, Algorithm 2)
 * and the over-relaxation of Section 5.2.
 *
 * Conventions for every entry point:
 *   - Return value: LPDEC_OK (0) or a negative LPDEC_E* status.  A
 *     human-readable message for the calling thread's last failure is
 *     available from lpdec_last_error().
 *   - "device pointer" means memory of the current CUDA device (cudaMalloc,
 *     a torch CUDA tensor, ...).  "host pointer" means ordinary CPU memory.
 *     The library never takes ownership of caller memory.
 *   - Decode calls that take a stream are stream-ordered and asynchronous:
 *     they return after enqueuing work on that stream; synchronize the stream
 *     before reading outputs.  stream == NULL means the legacy default stream.
 *   - All ADMM arithmetic on the GPU is FP32; FP64 is used there only to sum
 *     the per-frame residual norms of the stopping test.  The dual subgradient
 *     decoder (lpdec_decode_dual) works on integers, after computing each
 *     variable's Heaviside threshold ceil(-gamma_i/mu) once per frame in FP64.
 *   - Layouts are row-major: an LLR or x batch is [n_frames x n], frame f at
 *     element offset f*n.
 *   - Threads: decode calls on the same code from several host threads (and
 *     streams) are safe; they only read the code object.  The calls that change
 *     a code's tiles (lpdec_autotune, lpdec_set_tile, lpdec_set_streamed_tile,
 *     lpdec_dual_set_tile) must not run while another thread uses that code.
 */
#ifndef LPDEC_H
#define LPDEC_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define LPDEC_API __attribute__((visibility("default")))
#else
#define LPDEC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define LPDEC_OK        0
#define LPDEC_EINVAL   (-1) /* an argument is out of range or inconsistent */
#define LPDEC_ENOMEM   (-2) /* a host or device allocation failed, or a size limit is exceeded */
#define LPDEC_ECUDA    (-3) /* a CUDA runtime call failed (message has the CUDA error) */
#define LPDEC_ETIMEOUT (-4) /* a wait ran out of time before the result was ready */
#define LPDEC_EBUSY    (-5) /* a queue or budget is full; retry later */
#define LPDEC_ECLOSED  (-6) /* the object was shut down */

/* Per-frame iteration count written for a frame whose LLRs contain NaN/Inf:
 * that frame is not decoded (x = 0, bits = 0, cert = 0). */
#define LPDEC_FRAME_BAD_LLR (-1)

/* Per-frame iteration count written for a STREAMED frame abandoned because a
 * bounded wait on the movement of its parked state ran out (about 1 s), or
 * left unfinished after the last launch for that reason: its x, bits and
 * cert are not valid (cert = 0).  Not expected in normal operation. */
#define LPDEC_FRAME_ABANDONED (-2)

/* ---- storage type of the per-edge state --------------------------------- */
/* (The kernels keep w = z - lambda/mu and lambda/mu per edge; Algorithm 1's z
 * is w + lambda/mu.) */
#define LPDEC_STATE_F32  0
#define LPDEC_STATE_BF16 1 /* round-to-nearest-even on every store; FP32 arithmetic */
#define LPDEC_STATE_F16  2 /* round-to-nearest-even on every store; FP32 arithmetic */
#define LPDEC_STATE_Q16  3 /* 16-bit fixed point: k * s with k a 16-bit integer and s the smallest
                              power of two with 32767 s >= 1 + 6/mu (2^-13 at mu = 3), rounded to
                              nearest on every store; values beyond +-32767 s saturate.  FP32
                              arithmetic.  Uniform absolute precision: w and lambda/mu live in a
                              range of a few units, where BF16/FP16 lose low bits to the exponent. */

/* ---- schedules --------------------------------------------------------- */
#define LPDEC_SCHED_AUTO     0 /* RESIDENT when a frame's state fits in shared memory, else STREAMED */
#define LPDEC_SCHED_STREAMED 1 /* one kernel launch per ADMM iteration (or iters_per_launch); the
                                  edge state of every frame goes through device memory between
                                  launches */
#define LPDEC_SCHED_RESIDENT 2 /* one launch; each frame's z/lambda/x state stays in shared memory
                                  for all of its iterations */

typedef struct lpdec_code lpdec_code;     /* opaque: a parity-check matrix resident on one GPU */
typedef struct lpdec_server lpdec_server; /* opaque: a continuous-batching decode server */
typedef struct lpdec_mixed_plan lpdec_mixed_plan; /* opaque: a prepared mixed-code launch */

/* Decoder parameters (Algorithm 1 caption; Section 5.1 for the paper's defaults). */
typedef struct lpdec_params {
    double  mu;               /* ADMM penalty mu > 0 (eq. (augLag)) */
    double  rho;              /* over-relaxation rho in [1, 2) (Section 5.2) */
    double  eps;              /* stopping tolerance eps >= 0: stop when
                                 sum_j ||P_j x - z_j||^2 < eps^2 E and
                                 sum_j ||z_j - z_j^old||^2 < eps^2 E (E = number of edges;
                                 the paper's eps^2 M d for regular codes).
                                 eps = 0: run exactly max_iter iterations. */
    int32_t max_iter;         /* t_max >= 1 */
    int32_t state_dtype;      /* LPDEC_STATE_* */
    double  cert_tol;         /* certificate integrality tolerance, in (0, 0.5) */
    int32_t schedule;         /* LPDEC_SCHED_* */
    int32_t iters_per_launch; /* STREAMED only: ADMM iterations per kernel launch (>= 1) */
    int32_t reserved[6];      /* must be zero */
} lpdec_params;

/* Fill *p with the paper's Section 5.1 settings: mu = 3, rho = 1.9, eps = 1e-5,
 * max_iter = 1000, FP32 state, cert_tol = 1e-2, AUTO schedule, 1 iteration per launch. */
LPDEC_API void lpdec_params_default(lpdec_params *p);

/* Message describing the calling thread's most recent failure ("" if none). */
LPDEC_API const char *lpdec_last_error(void);

/* Library version string. */
LPDEC_API const char *lpdec_version(void);

/* ---- codes ------------------------------------------------------------- */

/*
 * Upload a parity-check matrix H (m x n) to the current CUDA device.
 * Section 2 defines H, the neighbourhoods N_c(j), N_v(i) and the selection
 * matrices P_j; the k-th edge of check j (in ascending column order) is the
 * k-th row of P_j.
 *   row_ptr[m+1], col_idx[E]: host pointers, H by rows (CSR); columns strictly
 *                             ascending within a row.
 *   col_ptr[n+1], row_idx[E]: host pointers, H by columns (CSC); rows strictly
 *                             ascending within a column.
 *   edge_perm[E]:             host pointer; edge_perm[t] is the CSR edge id of
 *                             CSC slot t.
 * The arrays are copied; the caller keeps ownership.
 * Errors: LPDEC_EINVAL if n or m <= 0, any check degree is 0 or > 32, any
 * variable degree is 0 (x_i is then undefined, Section 3.2), columns/rows are
 * unsorted or repeated, or the three layouts disagree; LPDEC_ENOMEM / LPDEC_ECUDA
 * on allocation or copy failure.  *out is set only on success.
 */
LPDEC_API int lpdec_code_create(int32_t n, int32_t m,
                      const int32_t *row_ptr, const int32_t *col_idx,
                      const int32_t *col_ptr, const int32_t *row_idx,
                      const int32_t *edge_perm, lpdec_code **out);

/* Shape of a code: n, m, number of edges E, largest check degree, and
 * k_rank = n - rank_GF(2)(H).  Any output pointer may be NULL. */
LPDEC_API int lpdec_code_info(const lpdec_code *code, int32_t *n, int32_t *m, int64_t *E,
                    int32_t *max_dc, int32_t *k_rank);

/* Free a code.  The caller must ensure no decode using it is still running. */
LPDEC_API int lpdec_code_destroy(lpdec_code *code);

/*
 * Autotuner: time the candidate tiles of a code (frames decoded at once per
 * CTA x threads per frame, within the register, barrier and shared-memory
 * limits) on the caller's sample of n_frames frames (llr: device pointer
 * [n_frames x n]) with params, keep the fastest for that state dtype and
 * schedule in the code object, and report it.  params.schedule = STREAMED
 * tunes the STREAMED tile (with params.max_iter launches per candidate, so a
 * few iterations suffice); its candidates include ring tiles (see
 * lpdec_set_streamed_tile), reported through lpdec_get_tile.  RESIDENT or AUTO
 * tunes the RESIDENT tile.  Later
 * decodes of the code use the tile of their schedule (STREAMED decodes fall
 * back to the RESIDENT tile when no STREAMED tile was tuned); the server and
 * lpdec_decode_mixed use the RESIDENT tile.
 * Synchronizes cuda_stream.  Any output pointer may be NULL.
 */
LPDEC_API int lpdec_autotune(lpdec_code *code, const lpdec_params *params, int32_t n_frames, const float *llr,
                             void *cuda_stream, int32_t *group_threads, int32_t *groups, double *ms_per_frame);

/* Set a code's tile for one state dtype by hand (groups x group_threads), for
 * both schedules; 0, 0 restores the built-in default.  group_threads is a
 * multiple of 32, groups <= 15, and a CTA holds at most 1024 threads (896 for
 * codes whose checks have degree 17..32, whose kernels are compiled for 896
 * threads to get more registers).  LPDEC_EINVAL for a tile that does not fit. */
LPDEC_API int lpdec_set_tile(lpdec_code *code, int32_t state_dtype, int32_t group_threads, int32_t groups);

/* Set a code's STREAMED tile for one state dtype by hand (the RESIDENT tile is
 * left as it is); 0, 0, 0 restores the fallback to the RESIDENT tile.
 * ring_slots = 0: the plain STREAMED kernel, each group loading its frame's
 * parked state into its own slice.  ring_slots = R > 0 (groups < R <= 64): a
 * producer warp per CTA (groups x group_threads + 32 threads) prefetches the
 * parked state of the next frames into a ring of R shared-memory slots while
 * the groups compute; results are identical.  LPDEC_EINVAL for a tile that
 * does not fit. */
LPDEC_API int lpdec_set_streamed_tile(lpdec_code *code, int32_t state_dtype, int32_t group_threads, int32_t groups,
                                      int32_t ring_slots);

/* The tile a decode of this code with this state dtype and schedule
 * (LPDEC_SCHED_*) would use now: tuned, set by hand, or the default;
 * ring_slots is 0 unless a STREAMED decode would run the ring kernel.  Any
 * output pointer may be NULL. */
LPDEC_API int lpdec_get_tile(const lpdec_code *code, int32_t state_dtype, int32_t schedule, int32_t *group_threads,
                             int32_t *groups, int32_t *ring_slots);

/* ---- decoding ---------------------------------------------------------- */

/*
 * Decode a batch of frames of one code: Algorithm 1 per frame.
 *   llr:       device pointer, [n_frames x n] FP32, gamma_i = log W(y_i|0)/W(y_i|1)
 *              (Section 2; positive favours bit 0).
 *   x_out:     device pointer, [n_frames x n] FP32: the x of the last iteration run.
 *   bits_out:  device pointer, [n_frames x n] uint8: b_i = [x_i > 1/2] (Section 5.1 rounding).
 *   iters_out: device pointer, [n_frames] int32: completed iterations when the stopping
 *              test first passed, or max_iter; LPDEC_FRAME_BAD_LLR for a frame with a
 *              non-finite LLR; LPDEC_FRAME_ABANDONED (STREAMED) for a frame whose
 *              state could not be moved in time.
 *   cert_out:  device pointer, [n_frames] uint8: 1 when the output is certified an ML
 *              codeword (Section 1: an integral LP optimum is the ML codeword):
 *              the residual test passes at the final iterate with tolerance
 *              max(eps, 1e-5), every x_i is within cert_tol of 0 or 1, and b
 *              satisfies every check.
 * Any of bits_out, iters_out, cert_out may be NULL.  n_frames == 0 is a no-op.
 * Errors (returned synchronously, before any work is queued): LPDEC_EINVAL for a
 * NULL code/llr/x_out, n_frames < 0, mu <= 0, rho outside [1, 2), eps < 0,
 * max_iter < 1, cert_tol outside (0, 0.5), an unknown state_dtype/schedule,
 * iters_per_launch < 1, or a RESIDENT schedule whose frame state does not fit
 * in shared memory; LPDEC_ENOMEM / LPDEC_ECUDA when workspace allocation or a
 * launch fails.  The call allocates its device workspace stream-ordered from
 * the library's memory pool (see lpdec_release_memory) and frees it the same
 * way.
 */
LPDEC_API int lpdec_decode(const lpdec_code *code, int32_t n_frames, const float *llr,
                 const lpdec_params *params, float *x_out, uint8_t *bits_out,
                 int32_t *iters_out, uint8_t *cert_out, void *cuda_stream);

/*
 * As lpdec_decode, but every buffer is a HOST pointer: the call copies llr to
 * the device, decodes, copies the outputs back and synchronizes the stream
 * before returning.  Outputs have the same meaning and shapes as above.
 * A batch of at least 8 waves (a wave: the frames the kernel holds in flight)
 * is cut into up to 8 chunks of whole waves, decoded alternately on
 * cuda_stream and an internal second stream so that the copies of one chunk
 * overlap the decode of its neighbours (results unchanged).  Page-locked host
 * buffers are needed for that overlap.
 */
LPDEC_API int lpdec_decode_host(const lpdec_code *code, int32_t n_frames, const float *llr,
                      const lpdec_params *params, float *x_out, uint8_t *bits_out,
                      int32_t *iters_out, uint8_t *cert_out, void *cuda_stream);

/*
 * Decode one batch whose frames belong to different codes (up to 8 codes, any
 * check degrees), in ONE persistent kernel launch: Algorithm 1 per frame with
 * per-frame early exit (eps > 0) and the RESIDENT schedule.  A CTA decodes
 * frames of one code at a time with that code's tile, and moves to another
 * code when the first runs out of frames, so early-exiting frames free their
 * slot for the next frame of any code.
 *   codes[n_codes]:     code handles, all on the current device.
 *   frame_code:         HOST pointer [n_frames]: the code index of each frame.
 *   llr, x_out, bits_out: device pointers; frames packed back to back in frame
 *                       order (frame f starts at sum_{g<f} n of code frame_code[g]).
 *   iters_out, cert_out: device pointers [n_frames] (may be NULL), as in lpdec_decode.
 * Results are identical to lpdec_decode of each code's frames alone.
 * Errors: LPDEC_EINVAL for n_codes outside [1, 8], NULL arguments, a frame_code
 * out of range, codes on different devices, the STREAMED schedule, or a code
 * whose frame state does not fit in shared memory; plus lpdec_decode's.
 */
LPDEC_API int lpdec_decode_mixed(const lpdec_code *const *codes, int32_t n_codes, int32_t n_frames,
                                 const int32_t *frame_code, const float *llr, const lpdec_params *params,
                                 float *x_out, uint8_t *bits_out, int32_t *iters_out, uint8_t *cert_out,
                                 void *cuda_stream);

/*
 * A prepared mixed-code decode, for batches whose composition repeats (the
 * same codes in the same frame order, new LLRs each time).
 *   lpdec_mixed_plan_create: validates like lpdec_decode_mixed, chooses the
 *       tiles, and copies the per-frame offsets and per-code frame lists to
 *       device memory it owns (synchronous; params are fixed for the plan).
 *   lpdec_mixed_plan_decode: queues one counter reset and ONE persistent kernel
 *       launch on cuda_stream, with buffers laid out as in lpdec_decode_mixed.
 *       It touches no host memory and allocates nothing, so it can be captured
 *       into a CUDA graph and replayed.  A plan serves one decode at a time.
 *   lpdec_mixed_plan_destroy: frees the plan (no decode may be in flight).
 */
LPDEC_API int lpdec_mixed_plan_create(const lpdec_code *const *codes, int32_t n_codes, int32_t n_frames,
                                      const int32_t *frame_code, const lpdec_params *params,
                                      lpdec_mixed_plan **out);
LPDEC_API int lpdec_mixed_plan_decode(lpdec_mixed_plan *plan, const float *llr, float *x_out, uint8_t *bits_out,
                                      int32_t *iters_out, uint8_t *cert_out, void *cuda_stream);
LPDEC_API int lpdec_mixed_plan_destroy(lpdec_mixed_plan *plan);

/*
 * As lpdec_decode, for callers that must not allocate device memory while they
 * run (for example a receive loop with a fixed memory footprint and a latency
 * budget that rules out allocator calls, or a host framework that owns all
 * device memory and forbids side allocations).  The paper has no counterpart:
 * this is a deployment variant of the same decode.
 *   - Scratch space comes from one fixed 32 MiB device array inside the library
 *     (held by every GPU that loads it, until the process exits) instead of
 *     cudaMallocAsync; the call itself never allocates or frees.
 *   - A decode that needs more scratch than 32 MiB is rejected with
 *     LPDEC_ENOMEM before any work is queued.  RESIDENT decodes need under 1 KiB;
 *     STREAMED decodes need about 2 * n_frames * E * (4 or 2) bytes.
 *   - The first call on each device looks up the array's device address (with
 *     that device current); make that first call before any stream capture.
 *   - Every call reuses the same array and clears the parts that must start at
 *     zero on its stream; two calls in flight on the GPU at the same time (on
 *     different streams, or from different threads) race on it, so serialize them.
 * Arguments, outputs and the other errors are those of lpdec_decode.
 */
LPDEC_API int lpdec_decode_noalloc(const lpdec_code *code, int32_t n_frames, const float *llr,
                                   const lpdec_params *params, float *x_out, uint8_t *bits_out,
                                   int32_t *iters_out, uint8_t *cert_out, void *cuda_stream);

/* ---- serving ----------------------------------------------------------- */

/*
 * A continuous-batching decode server on the current device.  Each code added
 * gets a pool of frame slots in device memory (LLRs, outputs and the z/lambda
 * state of frames in flight).  A scheduler thread, started by the first
 * submit, runs rounds for each code: admit queued frames into free slots,
 * advance every frame in flight by params.iters_per_launch ADMM iterations in
 * one launch, and retire frames that converged or reached max_iter (Algorithm 1
 * per frame, early exit by the stopping test).  Each code's rounds follow one
 * another on its own stream without waiting for the other codes' rounds.
 * Requests that arrive while a code's round is on the GPU join its next round.
 * A frame's result is identical to lpdec_decode of that frame alone.  While
 * rounds are in flight the scheduler thread polls their completion (it keeps
 * one host core busy, yielding it between polls); it sleeps when no frame is
 * queued or in flight.
 *   device_budget_bytes: upper bound on the device memory of all slot pools.
 *   cuda_stream: work already queued on this stream (NULL: the legacy default
 *                stream) completes before a code's first round; each code's
 *                rounds then run on a private stream, so codes overlap on the GPU.
 */
LPDEC_API int lpdec_server_create(size_t device_budget_bytes, void *cuda_stream, lpdec_server **out);

/* Register a code; *code_id indexes it in later submits.  The code must
 * outlive the server.  Codes may be added at any time, also while requests of
 * other codes are in flight; a new code joins the scheduler's next round. */
LPDEC_API int lpdec_server_add_code(lpdec_server *server, const lpdec_code *code, int32_t *code_id);

/*
 * Queue a request of n_frames frames of one code.  llr_host: HOST pointer
 * [n_frames x n], copied before the call returns.  The first request of a code
 * fixes that code's parameters and sizes its slot pool (min(4096, what is left
 * of the budget) slots); later requests of the code must pass the same
 * parameters.  Errors: LPDEC_EINVAL (bad arguments, different parameters),
 * LPDEC_ENOMEM (budget exhausted), LPDEC_EBUSY (too many frames queued),
 * LPDEC_ECLOSED (server shutting down), or the status of a failed scheduler.
 */
LPDEC_API int lpdec_server_submit(lpdec_server *server, int32_t code_id, int32_t n_frames, const float *llr_host,
                                  const lpdec_params *params, uint64_t *request_id);

/*
 * Wait up to timeout_ms (< 0: no limit) for a request; when done, copy its
 * outputs to the HOST buffers (any may be NULL; shapes as in lpdec_decode) and
 * release it (a request can be polled to completion once).  LPDEC_ETIMEOUT if
 * not done in time (the request stays queued); LPDEC_EINVAL for an unknown id.
 */
LPDEC_API int lpdec_server_poll(lpdec_server *server, uint64_t request_id, int32_t timeout_ms, float *x,
                                uint8_t *bits, int32_t *iters, uint8_t *cert);

/* Latency percentiles of completed requests (submit to completion, host clock),
 * decoded information bits per second since the first submit (design rate
 * k = n - m per frame), and frames completed.  Any pointer may be NULL. */
LPDEC_API int lpdec_server_stats(lpdec_server *server, double *p50_ms, double *p99_ms, double *bits_per_s,
                                 int64_t *frames);

/* Scheduler accounting: rounds run (of all codes), the host wall time of the
 * scheduler while a round was in flight, and the device time during which at
 * least one code's round was running (the union of the rounds' first-launch to
 * status-copy spans).  Any pointer may be NULL. */
LPDEC_API int lpdec_server_counters(lpdec_server *server, int64_t *rounds, double *round_wall_ms,
                                    double *round_gpu_ms);

/* Stop accepting requests, finish the frames already submitted, free the
 * server.  Calls racing with destroy on other threads get LPDEC_ECLOSED. */
LPDEC_API int lpdec_server_destroy(lpdec_server *server);

/*
 * Euclidean projection onto the parity polytope PP_d (Section 4.4, Algorithm 2)
 * of `count` vectors of dimension d, 1 <= d <= 32, computed exactly as the
 * decoder's check update computes it.
 *   v: device pointer [count x d] FP32 inputs;  z: device pointer [count x d] outputs.
 * Errors: LPDEC_EINVAL for d outside [1, 32], count < 0 or NULL pointers.
 */
LPDEC_API int lpdec_project(int32_t d, int64_t count, const float *v, float *z, void *cuda_stream);

/*
 * Device memory.  The decode calls allocate their device workspace and (host
 * entry points) buffers stream-ordered from one memory pool per device owned
 * by the library, which keeps freed memory for later calls instead of
 * returning it at each synchronization.  This call returns every pool's
 * unused memory to the driver; memory of calls still in flight stays.
 * Errors: LPDEC_ECUDA if a pool cannot be trimmed.
 */
LPDEC_API int lpdec_release_memory(void);

/*
 * Failure handling: the limit, in SM clock cycles, of the first wait of a
 * STREAMED launch on the bulk copies of a frame's parked state or on a ring
 * slot.  When such a wait runs out, the frame is marked LPDEC_FRAME_ABANDONED
 * and the group stops; the copies already in flight are then waited for with
 * the default limit, so the launch always ends with no copy outstanding.
 * clocks <= 0 restores the default, 2^31 cycles (about 1 s).  The paper has
 * no counterpart: the call exists so that the abandonment path can be
 * exercised (a tiny limit makes the waits run out) without faulting a GPU.
 * Process-wide; it applies to decodes queued after it.  Never fails.
 */
LPDEC_API int lpdec_set_wait_limit(int64_t clocks);

/* ---- dual subgradient decoding (appendix) ------------------------------- */

/*
 * Decode n_frames frames by dual subgradient ascent on the un-augmented
 * Lagrangian (the paper's appendix), for comparison with ADMM: from lambda = 0,
 * each iteration takes, from the same lambda^k,
 *   x_i = 1 if -gamma_i - sum_{j in N_v(i)} lambda_j^(i) > 0, else 0 (Heaviside),
 *   z_j = argmax_{z in PP_d} lambda_j^T z (Algorithm 3: the positive entries of
 *         lambda_j, and when they are odd in number, either the largest
 *         non-positive entry added, when it costs less than dropping the
 *         smallest positive entry, or that entry dropped; ties pick the lowest
 *         index and a tie between the two repairs drops),
 *   lambda_j += mu (P_j x - z_j),
 * until the subgradient P_j x - z_j vanishes on every check (then x is an
 * integral LP optimum, hence an ML codeword) or max_iter iterations ran.
 * Every decision is taken exactly (lambda is held as integer multiples of mu),
 * so the outputs equal an exact-arithmetic run of the method.
 *   code:      from lpdec_code_create, on the current device.
 *   llr:       device pointer, [n_frames x n] FP32 gamma, frame-major.
 *   mu:        step size, > 0 and finite.
 *   max_iter:  1 .. 32767.
 *   x_out:     device pointer, [n_frames x n] FP32: the final x (0 or 1).
 *   bits_out:  device pointer, [n_frames x n] uint8, or NULL: the same as bytes.
 *   iters_out: device pointer, [n_frames] int32, or NULL: iterations run;
 *              LPDEC_FRAME_BAD_LLR for a frame with a non-finite LLR (its x is 0).
 *   cert_out:  device pointer, [n_frames] uint8, or NULL: 1 when the
 *              subgradient vanished (the output is a certified LP optimum).
 * The call queues work on cuda_stream and returns; it allocates 4 bytes
 * stream-ordered.  Errors: LPDEC_EINVAL (NULL code, llr or x_out with
 * n_frames > 0, n_frames < 0, mu or max_iter out of range, a frame state that
 * does not fit in shared memory), LPDEC_ENOMEM / LPDEC_ECUDA from CUDA.
 */
LPDEC_API int lpdec_decode_dual(const lpdec_code *code, int32_t n_frames, const float *llr, double mu,
                                int32_t max_iter, float *x_out, uint8_t *bits_out, int32_t *iters_out,
                                uint8_t *cert_out, void *cuda_stream);

/* Tile of lpdec_decode_dual for this code: `groups` frames per CTA, each
 * decoded by `group_threads` threads (a multiple of 32; groups <= 15; at most
 * 1024 threads per CTA).  (0, 0) restores the built-in default.  LPDEC_EINVAL
 * for a tile outside those limits or one whose frame states exceed shared memory. */
LPDEC_API int lpdec_dual_set_tile(lpdec_code *code, int32_t group_threads, int32_t groups);

#ifdef __cplusplus
}
#endif

#endif /* LPDEC_H */
